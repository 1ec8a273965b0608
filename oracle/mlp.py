"""Oracle for the learned coefficient model -- TEST INFRASTRUCTURE.

A multilayer perceptron 3 -> 64 -> 64 -> 7 with SiLU activations stands in for the
transcendental parts of the thermal synchrotron coefficients of Sec. 2.5. Everything here is
plain numpy in float64: the definition of the seven learned quantities, the reconstruction of
the eight coefficients from them, the network's forward and backward passes, the loss and one
Adam step (Kingma & Ba 2015). With quant=True the forward and backward passes round the
operands of every matrix product to bfloat16 at the points where the tensor-core kernels do
(inputs, weights, hidden activations, back-propagated errors); sums stay exact.

Inputs (x = nu / nu_c with nu_c = (3/2) nu_B sin(theta) Theta_e^2, the variable of the fits):
  log10 x in [-3, 6], log10 Theta_e in [-1, 2], |cos theta_B| in [0, 1]
  mapped linearly to [-1, 1]; a fourth input fixed at 1 carries the first layer's bias.
Outputs (u = x^-1/3, X = (sqrt(2) 1e3 / (1.5 x))^1/2, z = 1 / Theta_e):
  o1 = ln[2.5651 (1 + 1.92 u + 0.9977 u^2)]        I_I(x) = exp(o1 - 1.8899 x^1/3)
  o2 = ln[2.5651 (1 + 0.932 u + 0.4998 u^2)]       I_Q(x) = exp(o2 - 1.8899 x^1/3)
  o3 = ln[1.8138/x + 3.423 u^2 + 0.02955 x^-1/2 + 2.0377 u]   I_V likewise
  o4 = f_m(X), o5 = g_m(X)                         Faraday conversion / rotation shapes
  o6 = ln(e^z K_2(z)),  o7 = ln(K_0(z) / K_2(z))   Maxwell-Juettner Bessel factors
  K_1/K_2 follows from K_2 = K_0 + (2/z) K_1. (Only the combination sin(theta) Theta^2 of
  pitch angle and temperature enters x; the cosine input is kept so that the model has the
  three inputs of the pitch-angle-resolved coefficients, and the fits make it redundant.)
Parameter vector (float, 4906 values): W1 [64][4] (column 3 = first-layer bias), W2 [64][64],
b2 [64], W3 [7][64], b3 [7], output offset [7], output scale [7], output trend A [7][3]. The
model is o = offset + scale * y + A f (f the three mapped inputs), y the network; offset, A and
scale are fixed before training: the least-squares affine fit of the targets on f and the
standard deviation of its residual, so that the network learns the non-linear remainder.
"""
from __future__ import annotations

import numpy as np

from . import bessel_kx, coefficients

N_IN, N_H, N_OUT = 3, 64, 7
LX_RANGE = (-3.0, 6.0)
LT_RANGE = (-1.0, 2.0)
OFF_W1, OFF_W2, OFF_B2, OFF_W3, OFF_B3, OFF_MEAN, OFF_SCALE, OFF_A = (0, 256, 4352, 4416, 4864,
                                                                     4871, 4878, 4885)
N_PARAMS = 4906

# CGS constants (CODATA 2018 / IAU nominal), the values the radiation oracle uses
_E = 4.80320471e-10
_ME = 9.1093837015e-28
_C = 2.99792458e10
_H = 6.62607015e-27


# ------------------------------------------------------------------ bfloat16 rounding
def bf16(a):
    """Round to the nearest bfloat16 (8 significant bits), ties to even, via float32."""
    f = np.asarray(a, dtype=np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


# ------------------------------------------------------------------ learned quantities
def fm(X):
    X = np.asarray(X, dtype=np.float64)
    return (2.011 * np.exp(-X ** 1.035 / 4.7) - np.cos(0.5 * X) * np.exp(-X ** 1.2 / 2.73)
            - 0.011 * np.exp(-X / 47.2))


def gm(X):
    return 1.0 - 0.11 * np.log(1.0 + 0.035 * np.asarray(X, dtype=np.float64))


def targets(lx, lt):
    """The seven learned quantities at log10 x, log10 Theta_e (arrays of equal shape)."""
    lx = np.asarray(lx, dtype=np.float64)
    lt = np.asarray(lt, dtype=np.float64)
    x = 10.0 ** lx
    u = x ** (-1.0 / 3.0)
    X = np.sqrt(np.sqrt(2.0) * 1.0e3 / (1.5 * x))
    o = np.empty(lx.shape + (N_OUT,))
    o[..., 0] = np.log(2.5651 * (1.0 + 1.92 * u + 0.9977 * u * u))
    o[..., 1] = np.log(2.5651 * (1.0 + 0.932 * u + 0.4998 * u * u))
    o[..., 2] = np.log(1.8138 / x + 3.423 * u * u + 0.02955 / np.sqrt(x) + 2.0377 * u)
    o[..., 3] = fm(X)
    o[..., 4] = gm(X)
    z = 1.0 / 10.0 ** lt
    k2 = np.vectorize(lambda zz: bessel_kx(2.0, zz))(z)
    k0 = np.vectorize(lambda zz: bessel_kx(0.0, zz))(z)
    o[..., 5] = np.log(k2)
    o[..., 6] = np.log(k0 / k2)
    return o


def model_inputs(theta_e, b_gauss, nu, cos_theta):
    """(log10 x, log10 Theta_e, |cos theta_B|) of one plasma sample; x is inf for sin = 0."""
    sth = np.sqrt(max(1.0 - cos_theta * cos_theta, 0.0))
    nub = _E * b_gauss / (2.0 * np.pi * _ME * _C)
    nuc = 1.5 * nub * sth * theta_e * theta_e
    lx = np.log10(nu / nuc) if nuc > 0.0 else np.inf
    return lx, np.log10(theta_e), abs(cos_theta)


def in_domain(lx, lt):
    return LX_RANGE[0] <= lx <= LX_RANGE[1] and LT_RANGE[0] <= lt <= LT_RANGE[1]


def reconstruct(o, ne, theta_e, b_gauss, nu, cos_theta):
    """The eight fluid-frame coefficients (j_I, j_Q, j_V, alpha_I, alpha_Q, alpha_V, rho_Q,
    rho_V) from the learned quantities o[7] and the exact closed-form prefactors."""
    out = np.zeros(8)
    if ne <= 0.0 or theta_e <= 0.0 or b_gauss <= 0.0:
        return out
    sth2 = 1.0 - cos_theta * cos_theta
    sth = np.sqrt(max(sth2, 0.0))
    nub = _E * b_gauss / (2.0 * np.pi * _ME * _C)
    z = 1.0 / theta_e
    x = nu / (1.5 * nub * sth * theta_e * theta_e)
    # exp(-1.8899 x^1/3) / K_2(z) = exp(-1.8899 x^1/3 + z - o6)
    ex = np.exp(-1.8899 * np.cbrt(x) + z - o[5])
    pre = ne * _E * _E * nu / (np.sqrt(3.0) * _C)
    out[0] = pre * np.exp(o[0]) * ex
    out[1] = pre * np.exp(o[1]) * ex
    out[2] = pre * 4.0 / (3.0 * theta_e) * (cos_theta / sth) * np.exp(o[2]) * ex
    hkt = _H * nu / (theta_e * _ME * _C * _C)
    inv_bnu = np.expm1(hkt) * _C * _C / (2.0 * _H * nu ** 3)
    out[3:6] = out[0:3] * inv_bnu
    k0_k2 = np.exp(o[6])
    k1_k2 = (1.0 - k0_k2) * z / 2.0
    base = ne * _E * _E / (_ME * _C)
    out[6] = base * nub * nub * sth2 / nu ** 3 * o[3] * (k1_k2 + 6.0 * theta_e)
    out[7] = 2.0 * base * nub * cos_theta / nu ** 2 * k0_k2 * o[4]
    return out


def exact_coefficients(ne, theta_e, b_gauss, nu, cos_theta):
    return coefficients(ne, theta_e, b_gauss, nu, cos_theta)


# ------------------------------------------------------------------ network
def features(lx, lt, c):
    """Network inputs [n][4]: the three inputs mapped to [-1, 1] and the constant 1."""
    lx, lt, c = (np.asarray(v, dtype=np.float64) for v in (lx, lt, c))
    f = np.empty(lx.shape + (4,))
    f[..., 0] = 2.0 * (lx - LX_RANGE[0]) / (LX_RANGE[1] - LX_RANGE[0]) - 1.0
    f[..., 1] = 2.0 * (lt - LT_RANGE[0]) / (LT_RANGE[1] - LT_RANGE[0]) - 1.0
    f[..., 2] = 2.0 * np.abs(c) - 1.0
    f[..., 3] = 1.0
    return f


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    return dict(W1=p[OFF_W1:OFF_W2].reshape(N_H, 4), W2=p[OFF_W2:OFF_B2].reshape(N_H, N_H),
                b2=p[OFF_B2:OFF_W3], W3=p[OFF_W3:OFF_B3].reshape(N_OUT, N_H),
                b3=p[OFF_B3:OFF_MEAN], mean=p[OFF_MEAN:OFF_SCALE], scale=p[OFF_SCALE:OFF_A],
                A=p[OFF_A:N_PARAMS].reshape(N_OUT, 3))


def pack(d):
    p = np.zeros(N_PARAMS)
    p[OFF_W1:OFF_W2] = np.ravel(d["W1"])
    p[OFF_W2:OFF_B2] = np.ravel(d["W2"])
    p[OFF_B2:OFF_W3] = d["b2"]
    p[OFF_W3:OFF_B3] = np.ravel(d["W3"])
    p[OFF_B3:OFF_MEAN] = d["b3"]
    p[OFF_MEAN:OFF_SCALE] = d["mean"]
    p[OFF_SCALE:OFF_A] = d["scale"]
    p[OFF_A:N_PARAMS] = np.ravel(d["A"])
    return p


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(p, F, quant=False):
    """Normalised outputs y [n][7] for network inputs F [n][4], with the intermediates."""
    d = unpack(p)
    q = bf16 if quant else (lambda a: np.asarray(a, dtype=np.float64))
    Fq = q(F)
    Z1 = Fq @ q(d["W1"]).T
    H1 = q(silu(Z1))
    Z2 = H1 @ q(d["W2"]).T + d["b2"]
    H2 = q(silu(Z2))
    Y = H2 @ q(d["W3"]).T + d["b3"]
    return Y, dict(F=Fq, Z1=Z1, H1=H1, Z2=Z2, H2=H2)


def trend(p, F):
    """offset + A f: the affine part of the model."""
    d = unpack(p)
    return d["mean"] + np.asarray(F, dtype=np.float64)[..., :3] @ d["A"].T


def outputs(p, F, quant=False):
    d = unpack(p)
    Y, _ = forward(p, F, quant)
    return trend(p, F) + d["scale"] * Y


def affine_normalisation(F, O):
    """offset, A and scale from targets O [n][7] at network inputs F [n][4]: least squares of
    O on (f, 1), scale = root mean square of its residual."""
    F = np.asarray(F, dtype=np.float64)
    beta, *_ = np.linalg.lstsq(F, np.asarray(O, dtype=np.float64), rcond=None)
    R = O - F @ beta
    return dict(mean=beta[3], A=beta[:3].T, scale=np.sqrt(np.mean(R * R, axis=0)))


def loss_and_grad(p, F, O, quant=False, n_total=None):
    """Mean squared error of the normalised outputs against targets O [n][7] (in o units),
    averaged over n_total samples x 7 outputs (default: this batch), and its gradient with
    respect to the parameter vector (zero for the fixed offset, scale and trend)."""
    d = unpack(p)
    q = bf16 if quant else (lambda a: np.asarray(a, dtype=np.float64))
    n = F.shape[0]
    n_total = n if n_total is None else n_total
    Y, c = forward(p, F, quant)
    T = (np.asarray(O, dtype=np.float64) - trend(p, F)) / d["scale"]
    E = Y - T
    loss = float(np.sum(E * E)) / (n_total * N_OUT)
    dY = 2.0 * E / (n_total * N_OUT)
    dYq = q(dY)
    # bias gradients are sums of the same (rounded) errors as the weight gradients: the
    # products carry a constant-1 operand row for them
    g = dict(W3=dYq.T @ c["H2"], b3=dYq.sum(axis=0))
    dH2 = dYq @ q(d["W3"])
    dZ2 = dH2 * silu_grad(c["Z2"])
    dZ2q = q(dZ2)
    g["W2"] = dZ2q.T @ c["H1"]
    g["b2"] = dZ2q.sum(axis=0)
    dH1 = dZ2q @ q(d["W2"])
    dZ1 = dH1 * silu_grad(c["Z1"])
    g["W1"] = q(dZ1).T @ c["F"]
    g["mean"] = np.zeros(N_OUT)
    g["scale"] = np.zeros(N_OUT)
    g["A"] = np.zeros((N_OUT, 3))
    return loss, pack(g)


def adam_step(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step number t >= 1) of every trained parameter; the output offset,
    scale and trend are left unchanged. Returns new (p, m, v)."""
    p, g, m, v = (np.array(a, dtype=np.float64) for a in (p, g, m, v))
    trained = np.zeros(N_PARAMS, dtype=bool)
    trained[:OFF_MEAN] = True
    m = np.where(trained, beta1 * m + (1.0 - beta1) * g, m)
    v = np.where(trained, beta2 * v + (1.0 - beta2) * g * g, v)
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    p = np.where(trained, p - lr * mh / (np.sqrt(vh) + eps), p)
    return p, m, v
