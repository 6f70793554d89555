"""Kernel matrices, pseudo-inverse and compressed M2L operators (oracle; FP64, plain numpy).

Test infrastructure: see the package docstring for who may import this module.
"""

from __future__ import annotations

import numpy as np

from . import geometry as G

FOUR_PI = 4.0 * np.pi


def laplace(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Dense kernel matrix K[i, j] = 1 / (4 pi |x_i - y_j|)  (Eq. 2, d = 3)."""
    d = x[:, None, :] - y[None, :, :]
    r = np.sqrt(np.sum(d * d, axis=-1))
    return 1.0 / (FOUR_PI * r)


def pinv_factors(A: np.ndarray, alpha: float = 0.0):
    """Backward-stable pseudo-inverse of Eqs. 7-10, kept as two factors.

    A = U S V^T (full SVD). Singular values above eps = (alpha + max(M, N) * eps_mach) * s_0
    are kept. Returns (V_eps, Ut_eps) with A^+ = V_eps @ Ut_eps and Ut_eps = S_eps^{-1} U_eps^T,
    which is the split storage the paper recommends (the footnote of Sec. 2.1.1).
    """
    U, s, Vt = np.linalg.svd(A, full_matrices=False)
    thresh = (alpha + max(A.shape) * np.finfo(np.float64).eps) * s[0]
    keep = s > thresh
    V_eps = Vt[keep].T.copy()
    Ut_eps = (U[:, keep] / s[keep][None, :]).T.copy()
    return V_eps, Ut_eps


def pinv_apply(factors, phi: np.ndarray) -> np.ndarray:
    """q = V_eps (Ut_eps phi) (Eq. 9); phi is (n_check, ...) with any trailing columns."""
    V_eps, Ut_eps = factors
    return V_eps @ (Ut_eps @ phi)


def down_pinv(p: int, level: int, root_width: float = 1.0, centre=None, p_c: int | None = None):
    """Factors of (K_tau)^+ for the downward check -> downward equivalent map at ``level``.

    Built from the actual surfaces of one box of that level (Sec. 2.2 notes this matrix is the
    same for every box of a level). ``p_c`` is the check surface's order (default p): with
    p_c > p the least-squares problem of Eq. 6 has more check than equivalent points.
    """
    w = G.box_width(level, root_width)
    c = np.zeros(3) if centre is None else np.asarray(centre, dtype=np.float64)
    x = G.surface_points(p if p_c is None else p_c, c, w, G.ALPHA_INNER)   # downward check
    y = G.surface_points(p, c, w, G.ALPHA_OUTER)   # downward equivalent
    return pinv_factors(laplace(x, y))


def up_pinv(p: int, level: int, root_width: float = 1.0, centre=None, p_c: int | None = None):
    """Factors of the upward check -> upward equivalent pseudo-inverse (Eq. 6 solved by Eq. 9)."""
    w = G.box_width(level, root_width)
    c = np.zeros(3) if centre is None else np.asarray(centre, dtype=np.float64)
    x = G.surface_points(p if p_c is None else p_c, c, w, G.ALPHA_OUTER)   # upward check
    y = G.surface_points(p, c, w, G.ALPHA_INNER)   # upward equivalent
    return pinv_factors(laplace(x, y))


def m2l_matrix(p: int, t, width: float = 1.0, p_c: int | None = None) -> np.ndarray:
    """K_t: downward check of a target at the origin vs upward equivalent of the source at t*width (Sec. 2.2)."""
    t = np.asarray(t, dtype=np.float64)
    x = G.surface_points(p if p_c is None else p_c, np.zeros(3), width, G.ALPHA_INNER)
    y = G.surface_points(p, t * width, width, G.ALPHA_INNER)
    return laplace(x, y)


def compressed_operators(p: int, rank_tol: float, width: float = 1.0, p_c: int | None = None):
    """SVD compression of Sec. 3.1 (Eqs. 12-14) over all 316 transfer vectors.

    K_fat = [K_1 ... K_316] ~ U Sigma V~^T and K_thin = [K_1; ...; K_316] ~ R~ Lambda S^T.
    The rank k keeps the singular values with s_i / s_0 >= rank_tol in either SVD (the larger
    of the two counts); rank_tol <= 0 keeps full rank (k = n). With a check order p_c > p the
    K_t are n_c x n and the two bases get their own ranks: U is n_c x k_c (K_fat's count, up to
    n_c), S is n x k (K_thin's, up to n) and C_t is k_c x k. ("k" is the equivalent-side rank,
    "kc" the check-side one; they are equal when p_c = p.)
    Returns dict(U (n,k), S (n,k), C (316,k,k), k, tvecs, s_fat, s_thin).
    """
    tv = G.transfer_vectors()
    Ks = np.stack([m2l_matrix(p, t, width, p_c) for t in tv])  # (316, n_c, n)
    n = Ks.shape[2]
    K_fat = np.concatenate(list(Ks), axis=1)               # n x 316 n
    K_thin = np.concatenate(list(Ks), axis=0)              # 316 n x n
    # Singular values and the n-dimensional singular vectors of the two stacked matrices.
    # For a tall A = Q R the SVD of R has the same singular values and right singular vectors,
    # so each SVD is taken of the n x n triangular factor (the left factor of K_fat is the right
    # factor of its transpose).
    _, s_fat, Ut_full = np.linalg.svd(np.linalg.qr(K_fat.T, mode="r"))
    U_full = Ut_full.T
    _, s_thin, St_full = np.linalg.svd(np.linalg.qr(K_thin, mode="r"))
    nc = Ks.shape[1]
    if rank_tol is None or rank_tol <= 0:
        kc, ke = nc, n
    else:
        k_fat = int(np.sum(s_fat / s_fat[0] >= rank_tol))
        k_thin = int(np.sum(s_thin / s_thin[0] >= rank_tol))
        if nc == n:
            kc = ke = max(k_fat, k_thin)   # equal orders: one k for both bases (Sec. 3.1)
        else:
            kc, ke = k_fat, k_thin         # check and equivalent spaces of different sizes
    U = U_full[:, :kc]
    S = St_full[:ke].T
    C = np.matmul(np.matmul(U.T[None], Ks), S[None])  # C_t = U^T K_t S  (kc x ke)
    return dict(U=U, S=S, C=C, k=ke, kc=kc, tvecs=tv, s_fat=s_fat, s_thin=s_thin, K=Ks)


def directional_operators(C: np.ndarray, dir_tol: float):
    """Directional recompression of Eq. 15: C_t ~ Ubar_t Sigmabar_t Vbar_t^T = Ubar_t Vbar'_t^T.

    For every transfer vector t the SVD of C_t keeps the k_t singular values with
    s_i >= dir_tol * s_0(C_t); dir_tol <= 0 keeps all k. Vbar'_t = Vbar_t Sigmabar_t is formed
    here, as Sec. 3.2 step 4 advises. Returns dict(Ubar: list of (k, k_t), Vbarp: list of
    (k, k_t), kt: (316,) ints, s: (316, k) singular values).
    """
    Ubar, Vbarp, kts, svals = [], [], [], []
    for Ct in C:
        Uc, sc, Vct = np.linalg.svd(Ct)
        kt = len(sc) if dir_tol is None or dir_tol <= 0 else int(np.sum(sc >= dir_tol * sc[0]))
        Ubar.append(Uc[:, :kt].copy())
        Vbarp.append((Vct[:kt].T * sc[:kt][None, :]).copy())
        kts.append(kt)
        svals.append(sc)
    return dict(Ubar=Ubar, Vbarp=Vbarp, kt=np.array(kts), s=np.array(svals))


def conv_grid_size(p: int) -> int:
    """Side of the convolution grid, 2P points (App. A.1)."""
    return 2 * p


def kernel_grid(p: int, t, width: float = 1.0, g: int | None = None) -> np.ndarray:
    """Circularly embedded kernel sequence for transfer vector t (App. A.1), real (g, g, g).

    For source lattice a and target lattice b the kernel value depends only on m = b - a in
    [-(p-1), p-1]^3:  G(m) = K(x_tau(b) - y_sigma(a)) = K(-t*w + h*m) with h = alpha*w/(p-1).
    G(m) is placed at index m mod g; all other entries are zero. With g >= 2p-1 the circular
    convolution of this grid with the zero-padded density equals the linear one at every
    surface point.
    """
    g = conv_grid_size(p) if g is None else g
    if g < 2 * p - 1:
        raise ValueError("convolution grid must have at least 2p-1 points per axis")
    t = np.asarray(t, dtype=np.float64)
    h = G.ALPHA_INNER * width / (p - 1)
    grid = np.zeros((g, g, g))
    r = np.arange(-(p - 1), p)
    mx, my, mz = np.meshgrid(r, r, r, indexing="ij")
    m = np.stack([mx, my, mz], axis=-1).reshape(-1, 3).astype(np.float64)
    d = -t[None, :] * width + h * m
    vals = 1.0 / (FOUR_PI * np.sqrt(np.sum(d * d, axis=-1)))
    mi = m.astype(np.int64) % g
    grid[mi[:, 0], mi[:, 1], mi[:, 2]] = vals
    return grid


def embed_density(p: int, q: np.ndarray, g: int | None = None) -> np.ndarray:
    """Place the n surface densities on the g^3 convolution grid at their lattice points (App. A.1)."""
    g = conv_grid_size(p) if g is None else g
    lat = G.surface_lattice(p)
    grid = np.zeros((g, g, g))
    grid[lat[:, 0], lat[:, 1], lat[:, 2]] = q
    return grid


def extract_surface(p: int, grid: np.ndarray) -> np.ndarray:
    lat = G.surface_lattice(p)
    return grid[lat[:, 0], lat[:, 1], lat[:, 2]]
