"""FP64 CPU oracle: every step of the sparsifying-preconditioned LS solve, written from the paper.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``): the product path never imports this.

Notation follows L. Ying, arXiv:1408.4495.  Grid: ``x_i = i h`` with ``i in {1..n}^d`` and
``h = 1/(n+1)`` (Sec. 2.1; the Laplace tables of Sec. 5 fix h = 1/(n+1)).  Arrays use the
0-based index ``a = i - 1`` in C order (last index fastest).  Offsets ``t`` are integer
d-tuples.  Complex numbers are numpy complex128 throughout.
"""

from __future__ import annotations

import itertools
import math

import numpy as np
import scipy.fft
import scipy.linalg
import scipy.sparse as sps
import scipy.sparse.linalg as spla
import scipy.special as sp

__all__ = [
    "grid_h", "grid_coords", "green", "k0_weight", "k0_corrected", "kernel_value", "kernel_table",
    "dense_K", "apply_K_direct", "apply_K_fft", "apply_operator", "plane_wave", "rhs",
    "point_class", "class_mu", "class_far_set", "stencil", "all_stencils",
    "assemble", "nd_order", "Preconditioner", "gmres_right", "solve",
    "check_buffer", "sparsity_ratio", "point_source", "laplace_solve", "far_field",
    "general_support", "general_apply", "general_rhs", "general_sketch", "general_stencils", "general_assemble",
    "general_solve",
]


# ----------------------------------------------------------------------------------------
# Sec. 2.1: grid, Green's function, Nystrom weights
# ----------------------------------------------------------------------------------------

def grid_h(n: int) -> float:
    """Step size h = 1/(n+1): n interior points per dimension of the unit cube (Sec. 2.1)."""
    return 1.0 / (n + 1)


def grid_coords(n: int, d: int):
    """Coordinates x_i = i h, i = 1..n, as d arrays of shape (n,)*d (Sec. 2.1)."""
    x = (np.arange(n, dtype=np.float64) + 1.0) * grid_h(n)
    return np.meshgrid(*([x] * d), indexing="ij")


def green(d: int, omega: float, r):
    """Free-space Green's function of -(Delta + omega^2) at distance r > 0 (Sec. 1):
    2D ``(i/4) H_0^(1)(omega r)``, 3D ``exp(i omega r) / (4 pi r)``.

    omega = 0 in 3D is the Laplace Green's function 1 / (4 pi r) of Sec. 5 (the same
    formula); the 2D Laplace kernel is not part of the paper and is refused."""
    r = np.asarray(r, dtype=np.float64)
    if d == 2:
        if omega == 0:
            raise ValueError("the Laplace variant (omega = 0) is three-dimensional (Sec. 5)")
        return 0.25j * sp.hankel1(0, omega * r)
    if d == 3:
        return np.exp(1j * omega * r) / (4.0 * np.pi * r)
    raise ValueError("d must be 2 or 3")


def k0_weight(d: int, omega: float, h: float) -> complex:
    """Weight k_0 of the singular point (Sec. 2.1).

    The paper states only that k_0 comes from a one-point correction of the trapezoidal
    rule.  Reading taken here: k_0 is the exact integral of G over the disk (2D) / ball
    (3D) centred at the origin whose area / volume equals the cell, h^d.

    2D, a = h / sqrt(pi):  int_0^a r H_0(omega r) dr = (a/omega) H_1(omega a) + 2i/(pi omega^2)
        so k_0 = (i pi a / (2 omega)) H_1^(1)(omega a) - 1/omega^2.
    3D, a = h (3/(4 pi))^(1/3):  int_0^a r e^{i omega r} dr
        so k_0 = e^{i omega a}(1/omega^2 - i a/omega) - 1/omega^2.
    3D Laplace (omega = 0, Sec. 5):  int_0^a (1/(4 pi r)) 4 pi r^2 dr = a^2 / 2, the
        omega -> 0 limit of the 3D form.
    """
    if d == 2:
        if omega == 0:
            raise ValueError("the Laplace variant (omega = 0) is three-dimensional (Sec. 5)")
        a = h / math.sqrt(math.pi)
        return complex(1j * math.pi * a / (2.0 * omega) * sp.hankel1(1, omega * a) - 1.0 / omega**2)
    if d == 3:
        a = h * (3.0 / (4.0 * math.pi)) ** (1.0 / 3.0)
        if omega == 0:
            return complex(a * a / 2.0)
        return complex(np.exp(1j * omega * a) * (1.0 / omega**2 - 1j * a / omega) - 1.0 / omega**2)
    raise ValueError("d must be 2 or 3")


def _radial_integral_G_gauss(d: int, omega: float, s: float) -> complex:
    """int over R^d of G(x) exp(-|x|^2 / (2 s^2)) dx, as a radial quadrature."""
    import scipy.integrate as si
    if d == 2:
        g = lambda r: 2 * math.pi * r * 0.25 * complex(-sp.y0(omega * r), sp.j0(omega * r))
    else:
        g = lambda r: r * complex(math.cos(omega * r), math.sin(omega * r))  # 4 pi r^2 / (4 pi r)
    w = lambda r: math.exp(-r * r / (2 * s * s))
    pts = [s * q for q in (0.25, 0.5, 1, 2, 4)]
    import warnings
    with warnings.catch_warnings():
        # quad may report roundoff near 1e-11 on the smooth J0 part; the convergence test
        # of k0_corrected checks the accuracy that matters
        warnings.simplefilter("ignore", si.IntegrationWarning)
        return _radial_quad(si, g, w, s, pts)


def _radial_quad(si, g, w, s, pts):
    re = si.quad(lambda r: g(r).real * w(r), 0, 12 * s, points=pts, limit=500, epsabs=0, epsrel=1e-11)[0]
    im = si.quad(lambda r: g(r).imag * w(r), 0, 12 * s, points=pts, limit=500, epsabs=0, epsrel=1e-11)[0]
    return complex(re, im)


def k0_corrected(d: int, omega: float, h: float, width: float = 8.0) -> complex:
    """One-point correction of the trapezoidal rule at the singular point (Sec. 2.1: accuracy
    O(h^4 log(1/h)) in 2D, citing Duan and Rokhlin; the weight is not printed).

    Reading: the corrected rule sum_{j != 0} G(h j) h^d f(h j) + k_0 f(0) must integrate
    G f for smooth f; its error for the plain trapezoidal sum is f(0) times a constant
    (depending on h, omega) plus O(h^4 log h) terms, so requiring exactness for one smooth
    radial f fixes k_0 to that order.  Here f is the Gaussian of width ``width`` h, the
    integral a radial quadrature and the lattice sum runs over |j| <= 11 width."""
    s = width * h
    M = int(math.ceil(11 * width))
    ax = np.arange(-M, M + 1)
    J = np.stack(np.meshgrid(*([ax] * d), indexing="ij"), -1).reshape(-1, d)
    J = J[np.any(J != 0, axis=1)]
    r = h * np.linalg.norm(J, axis=1)
    lattice = np.sum(green(d, omega, r) * h**d * np.exp(-r * r / (2 * s * s)))
    return complex(_radial_integral_G_gauss(d, omega, s) - lattice)


def kernel_value(d: int, omega: float, h: float, t, k0=None) -> np.ndarray:
    """k_t = G(h t) h^d for t != 0 and k_0 at t = 0 (Sec. 2.1, 2D and 3D forms).

    ``t`` is an integer array of shape (..., d); ``k0`` overrides the weight of the singular
    point (default: the ball integral of k0_weight; k0_corrected for the higher-order rule)."""
    t = np.asarray(t, dtype=np.float64)
    r = h * np.sqrt(np.sum(t * t, axis=-1))
    out = np.empty(r.shape, dtype=np.complex128)
    nz = r > 0
    out[nz] = green(d, omega, r[nz]) * h**d
    out[~nz] = k0_weight(d, omega, h) if k0 is None else k0
    return out


def kernel_table(n: int, d: int, omega: float, k0=None) -> np.ndarray:
    """Table of k_t for every t in (-n, n)^d, shape (2n-1,)*d, entry t stored at t + n - 1.

    These are all the offsets i - j between two grid points (Sec. 2.1, eq. lsd)."""
    t1 = np.arange(-(n - 1), n)
    T = np.stack(np.meshgrid(*([t1] * d), indexing="ij"), axis=-1)
    return kernel_value(d, omega, grid_h(n), T, k0)


# ----------------------------------------------------------------------------------------
# Sec. 2.1, eq. (lsd)/(lso): the discrete operator I + K omega^2 m
# ----------------------------------------------------------------------------------------

def _flat_index_offsets(n: int, d: int) -> np.ndarray:
    """All grid multi-indices in C order, shape (N, d)."""
    return np.stack(np.meshgrid(*([np.arange(n)] * d), indexing="ij"), axis=-1).reshape(-1, d)


def dense_K(ktab: np.ndarray, n: int, d: int) -> np.ndarray:
    """Dense N x N matrix K(i, j) = k_{i-j} (Sec. 2.1, after eq. lso).  Small n only."""
    idx = _flat_index_offsets(n, d)
    diff = idx[:, None, :] - idx[None, :, :] + (n - 1)
    return ktab[tuple(diff[..., a] for a in range(d))]


def apply_K_direct(ktab: np.ndarray, v: np.ndarray) -> np.ndarray:
    """(K v)_i = sum_j k_{i-j} v_j by direct summation of the definition (eq. lsd)."""
    n, d = v.shape[0], v.ndim
    return (dense_K(ktab, n, d) @ v.reshape(-1)).reshape(v.shape)


def apply_K_fft(ktab: np.ndarray, v: np.ndarray, workers: int | None = None) -> np.ndarray:
    """(K v) via the FFT (Sec. 1, third remark): the (2n)^d circulant embedding of k.

    k_t is placed at index t mod 2n for t in (-n, n)^d and the entries whose index has a
    component equal to n are zero; v is zero-padded to (2n)^d; the convolution restricted
    to the first n entries per dimension is exactly sum_j k_{i-j} v_j."""
    n, d = v.shape[0], v.ndim
    L = 2 * n
    kpad = np.zeros((L,) * d, dtype=np.complex128)
    src = np.arange(-(n - 1), n)
    dst = src % L
    kpad[np.ix_(*([dst] * d))] = ktab
    vpad = np.zeros((L,) * d, dtype=np.complex128)
    vpad[(slice(0, n),) * d] = v
    c = scipy.fft.ifftn(scipy.fft.fftn(kpad, workers=workers) * scipy.fft.fftn(vpad, workers=workers),
                        workers=workers)
    return c[(slice(0, n),) * d]


def apply_operator(ktab, omega: float, m: np.ndarray, u: np.ndarray, direct: bool = False,
                   workers: int | None = None) -> np.ndarray:
    """(I + K omega^2 m) u, eq. (lso)."""
    v = omega**2 * m * u
    Kv = apply_K_direct(ktab, v) if direct else apply_K_fft(ktab, v, workers)
    return u + Kv


def plane_wave(n: int, d: int, omega: float, direction) -> np.ndarray:
    """Incident plane wave u_I(x_i) = exp(i omega x_i . dir) on the grid (Sec. 3.3)."""
    X = grid_coords(n, d)
    phase = sum(X[a] * float(direction[a]) for a in range(d))
    return np.exp(1j * omega * phase)


def rhs(ktab, omega: float, m: np.ndarray, direction, direct: bool = False,
        workers: int | None = None) -> np.ndarray:
    """Discrete right-hand side g = K(-omega^2 m u_I) (eq. ls and eq. lsd).

    Reading: the paper calls g "the discretized value" of G * (-omega^2 m u_I); the same
    Nystrom weights k_t as the operator are used."""
    n, d = m.shape[0], m.ndim
    uI = plane_wave(n, d, omega, direction)
    v = -(omega**2) * m * uI
    return apply_K_direct(ktab, v) if direct else apply_K_fft(ktab, v, workers)


def point_source(ktab, n: int, d: int, point, strength: complex = 1.0) -> np.ndarray:
    """Right-hand side g = K f of Sec. 5 for a delta source of the given strength at the
    grid point ``point`` (0-based multi-index): the discrete delta is f_j = strength / h^d
    at j = point and 0 elsewhere (unit mass on the cell), so g_i = strength k_{i-point} / h^d."""
    f = np.zeros((n,) * d, dtype=np.complex128)
    f[tuple(point)] = strength / grid_h(n) ** d
    return apply_K_fft(ktab, f)


def far_field(n: int, d: int, omega: float, m: np.ndarray, u_total: np.ndarray, obs) -> np.ndarray:
    """Far-field pattern of the scattered field in the observation directions ``obs``
    (shape (k, d), unit vectors).  The scattered field is u_s = -K(omega^2 m u) (eq. ls with
    u the total field) and G(x - y) ~ c_d e^{i omega r} r^{-(d-1)/2} e^{-i omega theta . y}
    as r = |x| -> infinity in direction theta, so
        u_s(x) ~ e^{i omega r} r^{-(d-1)/2} u_inf(theta),
        u_inf(theta) = -c_d h^d sum_i e^{-i omega theta . x_i} omega^2 m_i u_i,
    c_2 = e^{i pi/4} / sqrt(8 pi omega) (large-argument form of (i/4) H_0^(1)),
    c_3 = 1 / (4 pi).  The discrete sum replaces the integral by the same quadrature as K."""
    X = grid_coords(n, d)
    h = grid_h(n)
    c = np.exp(1j * math.pi / 4) / math.sqrt(8 * math.pi * omega) if d == 2 else 1.0 / (4 * math.pi)
    v = (omega**2 * m * u_total).reshape(-1)
    out = np.empty(len(obs), dtype=np.complex128)
    for k, th in enumerate(obs):
        phase = sum(X[a] * float(th[a]) for a in range(d)).reshape(-1)
        out[k] = -c * h**d * np.sum(np.exp(-1j * omega * phase) * v)
    return out


def check_buffer(m: np.ndarray, b: int) -> bool:
    """m must vanish on the b+1 outermost layers of grid points (Sec. 2.1 and Sec. 3.1:
    a buffer of b layers next to the boundary layer).  Returns True when it does."""
    n, d = m.shape[0], m.ndim
    w = b + 1
    for a in range(d):
        lo = [slice(None)] * d
        hi = [slice(None)] * d
        lo[a] = slice(0, w)
        hi[a] = slice(n - w, n)
        if np.any(m[tuple(lo)] != 0) or np.any(m[tuple(hi)] != 0):
            return False
    return True


# ----------------------------------------------------------------------------------------
# Sec. 2.2 and Sec. 3.1: the sparsifying stencils A, B and C
# ----------------------------------------------------------------------------------------

def point_class(n: int, d: int) -> np.ndarray:
    """Class of every grid point, shape (n,)*d + (d,), entries in {-1, 0, +1} per dimension.

    -1: the point lies on the low face of that dimension (index 0), +1 on the high face
    (index n-1), 0 otherwise.  Class (0,..,0) is an interior point in the sense of Sec. 2.2
    (all of mu(i) lies in Omega); every other class is a boundary point."""
    idx = np.arange(n)
    c1 = np.where(idx == 0, -1, np.where(idx == n - 1, 1, 0))
    C = np.meshgrid(*([c1] * d), indexing="ij")
    return np.stack(C, axis=-1)


def class_mu(cls) -> list:
    """Translated neighbourhood mu(0) of a class (Sec. 2.2: ||i-j||_inf <= 1 inside Omega).

    Per dimension the offsets are {0, 1} on the low face, {-1, 0} on the high face and
    {-1, 0, 1} elsewhere.  Listed in C order."""
    per = [(0, 1) if c < 0 else (-1, 0) if c > 0 else (-1, 0, 1) for c in cls]
    return [tuple(t) for t in itertools.product(*per)]


def class_far_set(n: int, b: int, cls) -> np.ndarray:
    """The far set of a class (Sec. 3.1), shape (F, d).

    Interior (all zero): I_n = {-n < j_k < n} minus mu(0)  (eq. Fmin).
    Otherwise the product over dimensions of -n < j < -b (high face), b < j < n (low face,
    the mirror image) and -n < j < n (no face): E_n and C_n in 2D (eqs. Emin, Cmin) and
    F_n, E_n, C_n in 3D.  Reading: the 3D corner is printed at x_1 = 2; it is read as
    x_1 = 1 like every other face in that list."""
    d = len(cls)
    if all(c == 0 for c in cls):
        r = np.arange(-(n - 1), n)
        J = np.stack(np.meshgrid(*([r] * d), indexing="ij"), axis=-1).reshape(-1, d)
        keep = np.max(np.abs(J), axis=1) > 1
        return J[keep]
    per = []
    for c in cls:
        if c > 0:
            per.append(np.arange(-(n - 1), -b))
        elif c < 0:
            per.append(np.arange(b + 1, n))
        else:
            per.append(np.arange(-(n - 1), n))
    return np.stack(np.meshgrid(*per, indexing="ij"), axis=-1).reshape(-1, d)


def stencil(n: int, d: int, omega: float, b: int, cls, return_sigma: bool = False):
    """alpha for one class: min over |alpha| = 1 of |alpha K(mu(0), far)| (eqs. Fmin, Emin, Cmin).

    With K(mu(0), far) = U S V^*, alpha = U(:, |mu(0)|)^*, the conjugate of the left singular
    vector of the smallest singular value.  alpha is determined up to a unit factor;
    reading: it is normalised so that its centre coefficient (offset 0) is real and positive.
    Returns (mu, alpha[, singular values])."""
    h = grid_h(n)
    mu = class_mu(cls)
    far = class_far_set(n, b, cls)
    T = np.array(mu)[:, None, :] - far[None, :, :]          # K(t, j) = k_{t - j}
    Kmat = kernel_value(d, omega, h, T)
    U, S, _ = np.linalg.svd(Kmat, full_matrices=False)
    if S[-1] > 0 and S[-2] / S[-1] < 1.0 + 1e-8:
        raise ValueError("smallest singular value of K(mu, far) is not simple")
    alpha = np.conj(U[:, -1])
    centre = mu.index((0,) * d)
    ph = alpha[centre] / abs(alpha[centre])
    alpha = alpha / ph
    if return_sigma:
        return mu, alpha, S
    return mu, alpha


def all_stencils(n: int, d: int, omega: float, b: int = 2, k0=None):
    """alpha for all 3^d classes and C(i, mu(i)) = alpha K(mu(0), mu(0)) for the interior class.

    Sec. 2.2 defines C only for the interior rows (A); boundary rows of the preconditioner
    matrix are B alone (eq. PC).  ``k0`` overrides the weight of the singular point, which
    enters C only (the far sets exclude mu, so alpha never sees it).  Returns dict
    cls -> (mu, alpha), and (mu0, c)."""
    h = grid_h(n)
    out = {}
    for cls in itertools.product((-1, 0, 1), repeat=d):
        out[cls] = stencil(n, d, omega, b, cls)
    mu0, a0 = out[(0,) * d]
    T = np.array(mu0)[:, None, :] - np.array(mu0)[None, :, :]
    Kmm = kernel_value(d, omega, h, T, k0)                     # K(mu, mu)(t, t') = k_{t - t'}
    c = a0 @ Kmm                                               # C(0, t') = sum_t alpha_t k_{t-t'}
    return out, (mu0, c)


def assemble(n: int, d: int, omega: float, m: np.ndarray, sten, cint):
    """Sparse M = [A + C omega^2 m ; B] and S = [A ; B] (eqs. PC, ABop).

    Rows are kept in grid order rather than stacked interior-then-boundary; the
    preconditioner M^{-1} S is unchanged by a common row permutation.  Row i:
      S(i, i+t) = alpha_cls(i)(t)
      M(i, i+t) = alpha_cls(i)(t) + [i interior] c(t) omega^2 m_{i+t}."""
    N = n**d
    cls_arr = point_class(n, d)
    idx = np.arange(N).reshape((n,) * d)
    rows, cols, sv, mv = [], [], [], []
    mu0, c = cint
    cmap = dict(zip(mu0, c))
    w2m = omega**2 * m
    for cls, (mu, alpha) in sten.items():
        mask = np.all(cls_arr == np.array(cls), axis=-1)
        pts = np.argwhere(mask)                       # (P, d)
        if len(pts) == 0:
            continue
        interior = all(ci == 0 for ci in cls)
        for t, a in zip(mu, alpha):
            q = pts + np.array(t)
            r = idx[tuple(pts.T)]
            col = idx[tuple(q.T)]
            rows.append(r)
            cols.append(col)
            sv.append(np.full(len(r), a))
            if interior:
                mv.append(a + cmap[t] * w2m[tuple(q.T)])
            else:
                mv.append(np.full(len(r), a))
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    S = sps.csr_matrix((np.concatenate(sv), (rows, cols)), shape=(N, N))
    M = sps.csr_matrix((np.concatenate(mv), (rows, cols)), shape=(N, N))
    return M, S


# ----------------------------------------------------------------------------------------
# Sec. 2.2 / Sec. 3.2: nested dissection and the sparse solve of the preconditioner
# ----------------------------------------------------------------------------------------

def nd_order(n: int, d: int, leaf: int = 16) -> np.ndarray:
    """Geometric nested-dissection elimination order of the grid (Sec. 2.2, George 1973).

    A box is split along its longest side by a one-point-thick separator (the 3^d
    stencil couples only points at infinity-distance <= 1, so a slab of width 1 separates
    the two halves); the halves are ordered first, the separator last.  Boxes with at
    most ``leaf`` points are not split further."""
    idx = np.arange(n**d).reshape((n,) * d)
    out = []

    def rec(lo, hi):
        size = [hi[a] - lo[a] for a in range(d)]
        if min(size) <= 0:
            return
        if int(np.prod(size)) <= leaf or max(size) < 3:
            out.append(idx[tuple(slice(lo[a], hi[a]) for a in range(d))].reshape(-1))
            return
        ax = int(np.argmax(size))
        mid = (lo[ax] + hi[ax]) // 2
        hi1 = list(hi); hi1[ax] = mid
        lo2 = list(lo); lo2[ax] = mid + 1
        rec(lo, hi1)
        rec(lo2, hi)
        sl = [slice(lo[a], hi[a]) for a in range(d)]
        sl[ax] = slice(mid, mid + 1)
        out.append(idx[tuple(sl)].reshape(-1))

    rec([0] * d, [n] * d)
    return np.concatenate(out)


class Preconditioner:
    """u <= [A + C omega^2 m ; B]^{-1} [A ; B] g  (eq. PC).

    The sparse system is factored once with SuperLU (partial pivoting, FP64) after the
    symmetric nested-dissection permutation; each apply is one stencil product and one
    pair of triangular solves."""

    def __init__(self, M, S, n: int, d: int):
        self.M, self.S = M, S
        self.perm = nd_order(n, d)
        self.iperm = np.empty_like(self.perm)
        self.iperm[self.perm] = np.arange(len(self.perm))
        Mp = M[self.perm][:, self.perm].tocsc()
        self.lu = spla.splu(Mp, permc_spec="NATURAL")

    def solve_M(self, r: np.ndarray) -> np.ndarray:
        """M^{-1} r."""
        return self.lu.solve(r[self.perm])[self.iperm]

    def __call__(self, v: np.ndarray) -> np.ndarray:
        return self.solve_M(self.S @ v)


# ----------------------------------------------------------------------------------------
# Sec. 3.3: GMRES with relative tolerance 1e-6
# ----------------------------------------------------------------------------------------

def gmres_right(apply_A, apply_P, g: np.ndarray, tol: float = 1e-6, restart: int = 50,
                max_iter: int = 500):
    """Right-preconditioned restarted GMRES (Saad, Iterative Methods, Alg. 9.5) for A u = g.

    Reading: the paper names GMRES with relative tolerance 1e-6 but not the side of the
    preconditioner; right preconditioning makes the monitored quantity the true relative
    residual |g - A u| / |g|.  Modified Gram-Schmidt Arnoldi, complex Givens rotations.
    x0 = 0.  One iteration = one apply of P and one apply of A.
    Returns (u, iterations, relative residual history of the estimates)."""
    g = np.asarray(g, dtype=np.complex128).reshape(-1)
    N = g.size
    x = np.zeros(N, dtype=np.complex128)
    gnorm = np.linalg.norm(g)
    hist = []
    if gnorm == 0.0:
        return x, 0, hist
    total = 0
    while True:
        r = g - apply_A(x) if total > 0 else g.copy()
        beta = np.linalg.norm(r)
        if beta <= tol * gnorm or total >= max_iter:
            break
        V = [r / beta]
        Z = []
        H = np.zeros((restart + 1, restart), dtype=np.complex128)
        cs = np.zeros(restart, dtype=np.float64)
        sn = np.zeros(restart, dtype=np.complex128)
        s = np.zeros(restart + 1, dtype=np.complex128)
        s[0] = beta
        k = 0
        for j in range(restart):
            z = apply_P(V[j])
            w = apply_A(z)
            Z.append(z)
            total += 1
            for i in range(j + 1):
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            for i in range(j):
                a, bb = H[i, j], H[i + 1, j]
                H[i, j] = cs[i] * a + sn[i] * bb
                H[i + 1, j] = -np.conj(sn[i]) * a + cs[i] * bb
            a, bb = H[j, j], H[j + 1, j]
            rr = math.hypot(abs(a), abs(bb))
            if abs(a) == 0.0:
                cs[j], sn[j] = 0.0, 1.0
            else:
                cs[j] = abs(a) / rr
                sn[j] = (a / abs(a)) * np.conj(bb) / rr
            H[j, j] = cs[j] * a + sn[j] * bb
            H[j + 1, j] = 0.0
            s[j + 1] = -np.conj(sn[j]) * s[j]
            s[j] = cs[j] * s[j]
            k = j + 1
            res = abs(s[j + 1])
            hist.append(res / gnorm)
            hn = np.linalg.norm(w)
            if hn > 0:
                V.append(w / hn)
            if res <= tol * gnorm or total >= max_iter or hn == 0:
                break
        y = scipy.linalg.solve_triangular(H[:k, :k], s[:k])
        for i in range(k):
            x = x + y[i] * Z[i]
        if total >= max_iter:
            break
    return x, total, hist


def solve(n: int, d: int, omega: float, m: np.ndarray, directions, b: int = 2,
          tol: float = 1e-6, restart: int = 50, max_iter: int = 500, workers=None,
          precond: bool = True, k0=None):
    """The whole preconditioned solve for each incident direction (Secs. 2-3).

    ``k0`` overrides the weight of the singular point (default the ball integral of
    k0_weight; k0_corrected(d, omega, h) for the higher-order rule of Sec. 2.1); it enters
    the operator, the right-hand side and C.
    Returns dict with u (nrhs, n^d), iterations, true relative residuals, g."""
    if not check_buffer(m, b):
        raise ValueError("m must vanish within b+1 layers of the boundary")
    ktab = kernel_table(n, d, omega, k0)
    sten, cint = all_stencils(n, d, omega, b, k0)
    M, S = assemble(n, d, omega, m, sten, cint)
    P = Preconditioner(M, S, n, d)
    shape = (n,) * d

    def A(x):
        return apply_operator(ktab, omega, m, x.reshape(shape), workers=workers).reshape(-1)

    Pf = (lambda v: P(v)) if precond else (lambda v: v)
    us, its, res, gs = [], [], [], []
    for dr in directions:
        g = rhs(ktab, omega, m, dr, workers=workers).reshape(-1)
        u, it, _ = gmres_right(A, Pf, g, tol, restart, max_iter)
        gn = np.linalg.norm(g)
        res.append(np.linalg.norm(g - A(u)) / gn if gn > 0 else 0.0)
        us.append(u)
        its.append(it)
        gs.append(g)
    return dict(u=np.array(us), iters=its, resid=res, g=np.array(gs), P=P, ktab=ktab,
                sten=sten, cint=cint)


def laplace_solve(n: int, V: np.ndarray, points, b: int = 2, tol: float = 1e-6,
                  restart: int = 50, max_iter: int = 500, workers=None, strengths=None, k0=None):
    """Sec. 5: (I + K V) u = K f in 3D with the Laplace kernel k_t = h^3 / (4 pi h |t|),
    k_0 = a^2 / 2, and delta sources f at the given grid points.

    The sparsifying preconditioner is built exactly as in Secs. 2-3 from this kernel
    (Sec. 5 applies it without modification): the stencils are the SVD minimisers of
    K(mu, far) for the Laplace table, and M = [A + C V ; B].  The operator and M need only
    the product omega^2 m of the Helmholtz case, which is V here; the functions above are
    called with omega = 1 and m = V for those two steps and with omega = 0 for the kernel.
    ``k0`` overrides the weight of the singular point as in ``solve``.
    Returns dict with u (nsrc, n^3), iterations, true relative residuals, g."""
    d = 3
    V = np.asarray(V, dtype=np.float64)
    if not check_buffer(V, b):
        raise ValueError("V must vanish within b+1 layers of the boundary")
    ktab = kernel_table(n, d, 0.0, k0)
    sten, cint = all_stencils(n, d, 0.0, b, k0)
    M, S = assemble(n, d, 1.0, V, sten, cint)
    P = Preconditioner(M, S, n, d)
    shape = (n,) * d

    def A(x):
        return apply_operator(ktab, 1.0, V, x.reshape(shape), workers=workers).reshape(-1)

    us, its, res, gs = [], [], [], []
    for k, pt in enumerate(points):
        q = 1.0 if strengths is None else strengths[k]
        g = point_source(ktab, n, d, pt, q).reshape(-1)
        u, it, _ = gmres_right(A, P, g, tol, restart, max_iter)
        gn = np.linalg.norm(g)
        res.append(np.linalg.norm(g - A(u)) / gn if gn > 0 else 0.0)
        us.append(u)
        its.append(it)
        gs.append(g)
    return dict(u=np.array(us), iters=its, resid=res, g=np.array(gs), P=P, ktab=ktab,
                sten=sten, cint=cint)


# ----------------------------------------------------------------------------------------
# Sec. 4: general domains -- unknowns on the support of m only, randomized boundary stencils
# ----------------------------------------------------------------------------------------

def general_support(m: np.ndarray, b: int = 2) -> np.ndarray:
    """The unknowns of Sec. 4 as flat C-order indices: the grid points within infinity
    distance b + 1 of supp(m).

    Reading: Sec. 4 calls Omega "the support of m"; the boundary condition B(i, mu(i))
    (K omega^2 m)(mu(i), :) ~ 0 is the rectangular one of Sec. 3.1 only when m vanishes on
    the b + 1 layers next to the boundary (there the far sets leave out the b layers next to
    a face), so Omega is supp(m) surrounded by such a buffer, the counterpart of the
    rectangular buffer (reading 5).  Taking the bare support instead puts near-field columns
    with m != 0 into every boundary objective: measured on 3D n = 16, 24 that preconditioner
    needs 11-35 iterations against 3 with the buffer."""
    import scipy.ndimage as ndi
    mask = np.asarray(m) != 0
    se = np.ones((3,) * mask.ndim, dtype=bool)
    return np.flatnonzero(ndi.binary_dilation(mask, structure=se, iterations=b + 1).reshape(-1))


def general_apply(ktab, omega: float, m: np.ndarray, omega_idx, u_omega: np.ndarray) -> np.ndarray:
    """(I + K omega^2 m) restricted to Omega: u lives on the points omega_idx; K acts through
    the full grid with zeros outside Omega (m vanishes there, so nothing is lost)."""
    n, d = m.shape[0], m.ndim
    full = np.zeros(n**d, dtype=np.complex128)
    full[omega_idx] = u_omega
    v = (omega**2 * m.reshape(-1) * full).reshape((n,) * d)
    return u_omega + apply_K_fft(ktab, v).reshape(-1)[omega_idx]


def general_rhs(ktab, omega: float, m: np.ndarray, omega_idx, direction) -> np.ndarray:
    """g = K(-omega^2 m u_I) on Omega (reading 3 of the rectangular case)."""
    return rhs(ktab, omega, m, direction).reshape(-1)[omega_idx]


def general_sketch(n: int, d: int, omega: float, m: np.ndarray, R: np.ndarray, b: int = 2) -> np.ndarray:
    """The sketch T = (K omega^2 m) R of Sec. 4.1 on the unknowns Omega: R is |Omega| x r
    (rows in the order of general_support, zero outside Omega), one convolution of the
    definition per column, the rows of Omega kept.  Returns |Omega| x r."""
    idx = general_support(m, b)
    ktab = kernel_table(n, d, omega)
    T = np.empty((len(idx), R.shape[1]), dtype=np.complex128)
    for q in range(R.shape[1]):
        full = np.zeros(n**d, dtype=np.complex128)
        full[idx] = R[:, q]
        v = (omega**2 * m.reshape(-1) * full).reshape((n,) * d)
        T[:, q] = apply_K_fft(ktab, v).reshape(-1)[idx]
    return T


def general_stencils(n: int, d: int, omega: float, m: np.ndarray, R: np.ndarray, b: int = 2):
    """Stencils of Sec. 4.1.  Interior points of Omega (all 3^d neighbours in Omega) take the
    rectangular interior stencil alpha and C = alpha K(mu, mu) (Sec. 2.2 / 3.1, eq. Fmin).
    A boundary point i takes B(i, mu(i)) = alpha minimising |alpha T(mu(i), :)| over unit
    alpha, with T = (K omega^2 m) R for the Gaussian N x r matrix R (passed in, rows in the
    order of general_support), mu(i) = the neighbours of i (infinity distance <= 1) inside
    Omega: alpha = U(:, |mu(i)|)^* of T(mu(i), :) = U S V^*; reading as for the rectangular
    stencils: the coefficient at offset 0 made real and positive.
    Returns (omega_idx, interior mask over omega_idx, {point: (offsets, alpha)} for the
    boundary points, (mu0, alpha_int), (mu0, c))."""
    if not check_buffer(m, b):
        raise ValueError("m must vanish within b+1 layers of the grid boundary")
    idx = general_support(m, b)
    pos = -np.ones(n**d, dtype=np.int64)
    pos[idx] = np.arange(len(idx))
    T = general_sketch(n, d, omega, m, R, b)
    mu_all = [t for t in itertools.product((-1, 0, 1), repeat=d)]
    coords = np.stack(np.unravel_index(idx, (n,) * d), axis=-1)
    interior = np.zeros(len(idx), dtype=bool)
    bnd = {}
    for k, x in enumerate(coords):
        offs, rows = [], []
        for t in mu_all:
            y = x + np.array(t)
            if np.all(y >= 0) and np.all(y < n):
                j = pos[np.ravel_multi_index(tuple(y), (n,) * d)]
                if j >= 0:
                    offs.append(t)
                    rows.append(j)
        if len(offs) == len(mu_all):
            interior[k] = True
            continue
        U, S, _ = np.linalg.svd(T[rows], full_matrices=False)
        if len(S) > 1 and S[-1] > 0 and S[-2] / S[-1] < 1.0 + 1e-8:
            raise ValueError("smallest singular value of T(mu(i), :) is not simple")
        alpha = np.conj(U[:, -1])
        c0 = offs.index((0,) * d)
        alpha = alpha / (alpha[c0] / abs(alpha[c0]))
        bnd[int(idx[k])] = (offs, alpha)
    mu0, a0 = stencil(n, d, omega, b, (0,) * d)
    T2 = np.array(mu0)[:, None, :] - np.array(mu0)[None, :, :]
    c = a0 @ kernel_value(d, omega, grid_h(n), T2)                # C = alpha K(mu, mu)
    return idx, interior, bnd, (mu0, a0), (mu0, c)


def general_assemble(n: int, d: int, omega: float, m: np.ndarray, stencils):
    """Sparse M = [A + C omega^2 m ; B] and S = [A ; B] on Omega (eq. PC with the stencils of
    general_stencils), rows and columns in the order of general_support."""
    idx, interior, bnd, (mu0, a0), (mu0c, c) = stencils
    pos = -np.ones(n**d, dtype=np.int64)
    pos[idx] = np.arange(len(idx))
    amap, cmap = dict(zip(mu0, a0)), dict(zip(mu0c, c))
    w2m = (omega**2 * m).reshape(-1)
    rows, cols, sv, mv = [], [], [], []
    for k, i in enumerate(idx):
        x = np.array(np.unravel_index(i, (n,) * d))
        if interior[k]:
            offs, alpha = mu0, [amap[t] for t in mu0]
        else:
            offs, alpha = bnd[int(i)]
        for t, a in zip(offs, alpha):
            j = int(np.ravel_multi_index(tuple(x + np.array(t)), (n,) * d))
            rows.append(k)
            cols.append(pos[j])
            sv.append(a)
            mv.append(a + cmap[t] * w2m[j] if interior[k] else a)
    N = len(idx)
    S = sps.csr_matrix((np.array(sv), (rows, cols)), shape=(N, N))
    M = sps.csr_matrix((np.array(mv), (rows, cols)), shape=(N, N))
    return M, S


def general_solve(n: int, d: int, omega: float, m: np.ndarray, directions, R: np.ndarray, b: int = 2,
                  tol: float = 1e-6, restart: int = 50, max_iter: int = 500):
    """The whole Sec. 4 solve for each incident direction: GMRES on (I + K omega^2 m) u = g
    restricted to Omega, right-preconditioned with [A + C omega^2 m ; B]^{-1} [A ; B] built
    from general_stencils (sparse LU with SuperLU's column ordering).
    Returns dict with omega_idx, u (nrhs, |Omega|), iterations, true relative residuals, g."""
    ktab = kernel_table(n, d, omega)
    st = general_stencils(n, d, omega, m, R, b)
    idx = st[0]
    M, S = general_assemble(n, d, omega, m, st)
    lu = spla.splu(M.tocsc())

    def A(x):
        return general_apply(ktab, omega, m, idx, x)

    def P(v):
        return lu.solve(S @ v)

    us, its, res, gs = [], [], [], []
    for dr in directions:
        g = general_rhs(ktab, omega, m, idx, dr)
        u, it, _ = gmres_right(A, P, g, tol, restart, max_iter)
        gn = np.linalg.norm(g)
        res.append(np.linalg.norm(g - A(u)) / gn if gn > 0 else 0.0)
        us.append(u)
        its.append(it)
        gs.append(g)
    return dict(omega_idx=idx, u=np.array(us), iters=its, resid=res, g=np.array(gs), stencils=st)


def sparsity_ratio(n: int, d: int, omega: float, b: int = 2) -> float:
    """max over far j of |(A K)(i, j)| divided by max |C(i, mu(i))| for an interior row
    (the approximation A K ~ C of Sec. 2.2).  Reported only: the paper prints no value."""
    h = grid_h(n)
    mu, alpha = stencil(n, d, omega, b, (0,) * d)
    far = class_far_set(n, b, (0,) * d)
    T = np.array(mu)[:, None, :] - far[None, :, :]
    off = alpha @ kernel_value(d, omega, h, T)
    T2 = np.array(mu)[:, None, :] - np.array(mu)[None, :, :]
    on = alpha @ kernel_value(d, omega, h, T2)
    return float(np.max(np.abs(off)) / np.max(np.abs(on)))
