"""Independent pins of an s-Gaussian integral routine (S, T, V, W0 of Sec. II, Eqs. 4-7).

Every check takes the routine under test as a callable
    ints(nuc_xyz (L, 3), nuc_z (L,), bf_xyz (n, 3), bf_alpha (n,)) -> dict S, T, V, W0 (n x n)
and compares it with something that does not share its formulas:

* one-centre closed forms (every element, relative 1e-13);
* the Boys function F0 through scipy's regularised incomplete gamma function, on one-centre
  pairs whose nucleus is displaced so that p |P - C|^2 spans 0 .. 1e4 (both evaluation
  branches of any implementation; V relative 1e-13);
* V of a whole cluster, element by element, from the textbook Gaussian-product closed form
  with the same scipy Boys function (relative 1e-12 on every element above the floor
  1e-290, i.e. every element that does not underflow);
* T = 1/2 sum_k d2 S / dA_k dB_k and W0 = sum_k d2 V / dA_k dB_k (their definitions as
  gradients of the basis functions) by central differences of the routine's own S and V at
  displaced centres, Richardson-extrapolated; on sampled pairs (relative 1e-7) and, for W0,
  on every element of a cluster with a step chosen per element from its exponents and
  centre distance (2e-7 of max(|W0|, r^2 |V|), r the element's inverse length scale);
* V by 1D quadrature of the Gaussian transform of 1/r (no Boys function; relative 1e-11).

None of these uses the workload generator's integral code."""
import numpy as np
from scipy import integrate, special

PI = np.pi


def boys0_scipy(T):
    """F0(T) = int_0^1 exp(-T t^2) dt via the regularised lower incomplete gamma function."""
    T = np.asarray(T, dtype=np.float64)
    out = np.ones_like(T)
    nz = T > 0
    out[nz] = special.gamma(0.5) * special.gammainc(0.5, T[nz]) / (2.0 * np.sqrt(T[nz]))
    return out


def closed_form_STV(nuc_xyz, nuc_z, bf_xyz, bf_alpha):
    """Textbook S, T, V over normalised s primitives (Gaussian product theorem), with the
    scipy Boys function."""
    a = bf_alpha[:, None]
    b = bf_alpha[None, :]
    p = a + b
    mu = a * b / p
    AB2 = ((bf_xyz[:, None, :] - bf_xyz[None, :, :]) ** 2).sum(-1)
    K = (4 * a * b / PI**2) ** 0.75 * np.exp(-mu * AB2)
    S = K * (PI / p) ** 1.5
    T = mu * (3 - 2 * mu * AB2) * S
    P = (a[..., None] * bf_xyz[:, None, :] + b[..., None] * bf_xyz[None, :, :]) / p[..., None]
    V = np.zeros_like(S)
    for C, Z in zip(nuc_xyz, nuc_z):
        V -= Z * K * (2 * PI / p) * boys0_scipy(p * ((P - C) ** 2).sum(-1))
    return S, T, V


def check_one_centre(ints):
    al = 0.01 * 2.0 ** np.arange(0, 30, 3)
    n = len(al)
    Z = 47.0
    I = ints(np.zeros((1, 3)), np.array([Z]), np.zeros((n, 3)), al)
    a, b = np.meshgrid(al, al, indexing="ij")
    p = a + b
    Na, Nb = (2 * a / PI) ** 0.75, (2 * b / PI) ** 0.75
    ref = {"S": (2 * np.sqrt(a * b) / p) ** 1.5}
    ref["T"] = 3 * a * b / p * ref["S"]
    ref["V"] = -Z * Na * Nb * 2 * PI / p
    # W0 = 4ab <g_a| r^2 (-Z/r) |g_b> = -4abZ Na Nb 4pi / (2 p^2)
    ref["W0"] = -8 * PI * a * b * Z * Na * Nb / p**2
    for k, r in ref.items():
        assert np.allclose(I[k], r, rtol=1e-13, atol=0), k


def check_boys_through_V(ints):
    """One-centre pairs (both functions at the origin) with a nucleus at distance d: every
    V element is -Z Na Nb (2 pi / p) F0(p d^2)."""
    al = np.array([0.05, 0.3, 1.0, 4.0, 30.0, 500.0])
    n = len(al)
    for d in (0.0, 1e-4, 0.05, 0.3, 0.9, 1.7, 2.6, 4.0):
        I = ints(np.array([[0.0, 0.0, d]]), np.array([3.0]), np.zeros((n, 3)), al, )
        a, b = np.meshgrid(al, al, indexing="ij")
        p = a + b
        ref = -3.0 * (2 * a / PI) ** 0.75 * (2 * b / PI) ** 0.75 * 2 * PI / p * boys0_scipy(p * d * d)
        assert np.allclose(I["V"], ref, rtol=1e-13, atol=0), d
    # the arguments covered: from 0 to about 1e4
    assert (2 * al.max() * 4.0**2) > 1e4


def check_elementwise_V(ints, nuc_xyz, nuc_z, bf_xyz, bf_alpha, floor=1e-290):
    I = ints(nuc_xyz, nuc_z, bf_xyz, bf_alpha)
    S, T, V = closed_form_STV(nuc_xyz, nuc_z, bf_xyz, bf_alpha)
    for k, ref in (("S", S), ("T", T), ("V", V)):
        got = I[k]
        assert np.array_equal(got, got.T), k
        big = np.abs(ref) > floor
        rel = np.abs(got[big] - ref[big]) / np.abs(ref[big])
        assert rel.max() <= 1e-12, (k, rel.max())
        # below the floor both sides must be tiny too
        assert np.all(np.abs(got[~big]) <= 1e-280), k
    return I


def _displaced_block(ints, nuc_xyz, nuc_z, xa, aa, xb, ab):
    """Off-diagonal block [rows = functions (xa, aa), cols = (xb, ab)] of one call."""
    I = ints(nuc_xyz, nuc_z, np.concatenate([xa, xb]), np.concatenate([aa, ab]))
    na = len(aa)
    return {k: v[:na, na:] for k, v in I.items()}


def mixed_derivative(ints, key, nuc_xyz, nuc_z, xa, aa, xb, ab, h):
    """sum_k d2 M / dA_k dB_k of the block M[key] by central differences with step h (an
    array broadcastable to the block), Richardson-extrapolated from h and 2h."""

    def D(step):
        tot = 0.0
        for k in range(3):
            e = np.zeros(3)
            e[k] = step
            f = lambda sa, sb: _displaced_block(ints, nuc_xyz, nuc_z, xa + sa * e, aa, xb + sb * e, ab)[key]
            tot = tot + (f(1, 1) - f(1, -1) - f(-1, 1) + f(-1, -1)) / (4 * step * step)
        return tot

    return (4 * D(h) - D(2 * h)) / 3


def check_finite_differences(ints):
    nuc = np.array([[0.0, 0.0, 0.0], [1.1, -0.7, 0.2], [-2.0, 3.0, 9.0]])
    Zs = np.array([3.0, 2.0, 47.0])
    A = np.array([[0.1, -0.2, 0.3]])
    B = np.array([[0.6, 0.4, -0.5]])
    for a, b in ((0.7, 1.3), (0.2, 3.0), (2.5, 2.5), (0.05, 0.4)):
        aa, ab = np.array([a]), np.array([b])
        I = _displaced_block(ints, nuc, Zs, A, aa, B, ab)
        fdS = mixed_derivative(ints, "S", nuc, Zs, A, aa, B, ab, 1e-3)
        fdV = mixed_derivative(ints, "V", nuc, Zs, A, aa, B, ab, 1e-3)
        assert abs(I["T"][0, 0] - 0.5 * fdS[0, 0]) <= 1e-7 * abs(I["T"][0, 0]), (a, b)
        assert abs(I["W0"][0, 0] - fdV[0, 0]) <= 1e-7 * abs(I["W0"][0, 0]), (a, b)


def check_W0_elementwise_fd(ints, nuc_xyz, nuc_z, bf_xyz, bf_alpha, floor=1e-250):
    """W0 of every element against the mixed second derivative of V, with a step per
    element: V_ab varies on the length scale 1/r, r = max(sqrt(a + b), 2 mu |A - B|) (the
    width of the Gaussian product and the slope of its prefactor exp(-mu |A - B|^2)), and the
    step is h = 0.01 / r, taken from a ladder of steps."""
    n = len(bf_alpha)
    I = ints(nuc_xyz, nuc_z, bf_xyz, bf_alpha)
    a, b = bf_alpha[:, None], bf_alpha[None, :]
    p = a + b
    R = np.sqrt(((bf_xyz[:, None, :] - bf_xyz[None, :, :]) ** 2).sum(-1))
    r = np.maximum(np.sqrt(p), 2 * a * b / p * R)
    ladder = 0.01 / np.geomspace(r.min(), r.max(), 24)
    pick = np.abs(np.log(0.01 / r)[..., None] - np.log(ladder)).argmin(-1)
    fd = np.zeros((n, n))
    for i, h in enumerate(ladder):
        sel = pick == i
        if sel.any():
            fd[sel] = mixed_derivative(ints, "V", nuc_xyz, nuc_z, bf_xyz, bf_alpha, bf_xyz, bf_alpha, h)[sel]
    W0 = I["W0"]
    # the difference quotient's scale: r^2 |V| (each derivative brings down about r)
    scale = np.maximum(np.abs(W0), r * r * np.abs(I["V"]))
    big = scale > floor
    err = np.abs(fd - W0)[big] / scale[big]
    assert err.max() <= 2e-7, err.max()


def check_quadrature(ints):
    """V_ab = -sum_C Z_C (2/sqrt(pi)) int_0^inf <g_a| exp(-u^2 |r - C|^2) |g_b> du."""
    nuc = np.array([[-0.5, 0.7, 0.6], [1.3, 0.2, -0.8]])
    Zs = np.array([5.0, 2.0])
    A, B = np.array([0.0, 0.0, 0.0]), np.array([0.9, 0.3, -0.4])
    for a, b in ((0.8, 0.35), (3.0, 0.1), (0.02, 0.05)):
        Na, Nb = (2 * a / PI) ** 0.75, (2 * b / PI) ** 0.75
        ref = 0.0
        for C, Z in zip(nuc, Zs):
            def overlap3(u):
                c = u * u
                q = a + b + c
                P = (a * A + b * B + c * C) / q
                ex = a * A @ A + b * B @ B + c * C @ C - q * P @ P
                return Na * Nb * (PI / q) ** 1.5 * np.exp(-ex)

            val, _ = integrate.quad(overlap3, 0, np.inf, epsabs=0, epsrel=1e-13, limit=400)
            ref -= Z * 2 / np.sqrt(PI) * val
        got = _displaced_block(ints, nuc, Zs, A[None], np.array([a]), B[None], np.array([b]))["V"][0, 0]
        assert abs(got - ref) <= 1e-11 * abs(ref), (a, b, got, ref)
