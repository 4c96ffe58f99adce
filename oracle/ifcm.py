"""FP64 reference of the IFCM step function of 3DPIFCM (Eqs 1-10).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Plain numpy in
float64: every voxel loop of the paper is written as one whole-array
operation per neighbour offset, with no blocking, fusion or reordering
beyond what the equations state.

Layout: a volume ``x`` has shape (nz, ny, nx); memberships ``U`` have shape
(c, nz, ny, nx); centres ``C`` have shape (c,).  A 2D image is nz = 1.

Readings of points the paper leaves open (the paper's equation in brackets):

R1 [Eq 7, Eq 8]  q^2_ik in Eq 7 is the squared Euclidean offset of Eq 8
                 (dx^2 + dy^2 + dz^2), so face / edge / corner neighbours
                 weigh 1 / 2 / 3.
R2 [Eq 2, Eq 4]  1 - lambda*H - xi*F can be negative for lambda, xi in
                 [0, 1]; it is clamped at 0 and d^2 is floored at
                 ``dist_floor`` (1e-12) so that Eq 2 stays defined.
R3 [Eq 5]        where sum_k g_ik = 0 (every neighbour equals x_i) the
                 shell's H term is the plain mean of u_kj over the shell (the
                 limit of equal weights).  A shell with no in-volume voxel
                 drops out and W is renormalised over the remaining shells;
                 with none left H = F = 0.
R4 [Eq 9]        neighbours outside the volume are excluded (no padding).
R5 [Alg 1 s4]    one fitness evaluation runs IFCM from the shared FCM start
                 (U0, C0) until max|du| < eps or max_iter iterations; the
                 fitness is the J of the last iteration.
R6 [Alg 2 s6-8]  H and F of iteration t use U^t (Jacobi order).
R7 [Eq 1]        J^t is evaluated with the d^2 that produced U^{t+1}, i.e.
                 J^t = sum_ij (u^{t+1}_ij)^m d^2_ij(C^t, H(U^t), F(U^t)).
R10 [Alg 1 s2]   the unspecified "Modified_FCM with Gaussian mixture
                 model" start is replaced by plain FCM (lambda = xi = 0)
                 from c_j = (j + 1/2)/c and u_ij = 1/c.
Shells [Eq 9, Eq 10]  NB is the set of Eq 9 (L = 3: the 26 voxels around
                 x_i in 3D, 8 in 2D); shell S_r holds the members at
                 Chebyshev distance r, r = 1..V, with W_r of Eq 10.
R17 [Eq 9, Eq 10]  Eq 10 makes V "the distance of the furthest voxel", but
                 Eq 9's ball with L = 3 holds only distance-1 voxels.  For V
                 shells L is the smallest value whose ball contains the whole
                 cube of Chebyshev radius V (2^(L-1) > 3 V^2): L = 3 for V = 1,
                 5 for V = 2, 6 for V = 3.  The neighbourhood is that
                 cube without its centre, and S_r is its shell at distance r.
"""
import math

import numpy as np


# --------------------------------------------------------------------------
# Algorithm 2 step 1: min-max normalisation over the whole volume
# --------------------------------------------------------------------------
def normalize(vol):
    """x <- (x - min) / (max - min) over the entire volume (Alg 2 step 1)."""
    v = np.asarray(vol, dtype=np.float64)
    if v.size == 0 or not np.all(np.isfinite(v)):
        raise ValueError("volume is empty or holds NaN/Inf")
    lo, hi = v.min(), v.max()
    if hi == lo:
        raise ValueError("constant volume: max == min")
    return (v - lo) / (hi - lo)


# --------------------------------------------------------------------------
# Eq 9 (neighbourhood), Eq 10 (shell weights)
# --------------------------------------------------------------------------
def cube_L(V):
    """Smallest L of Eq 9 whose ball holds the cube of Chebyshev radius V
    (reading R17): 2^(L-1) > 3 V^2."""
    L = 1
    while 2 ** (L - 1) <= 3 * V * V:
        L += 1
    return L


def neighbourhood(L=3):
    """Offsets (dz, dy, dx) with 0 < dx^2 + dy^2 + dz^2 < 2^(L-1)  (Eq 9)."""
    bound = 2 ** (L - 1)
    reach = int(math.isqrt(bound)) + 1
    offs = []
    for dz in range(-reach, reach + 1):
        for dy in range(-reach, reach + 1):
            for dx in range(-reach, reach + 1):
                s = dx * dx + dy * dy + dz * dz
                if 0 < s < bound:
                    offs.append((dz, dy, dx))
    return offs


def shells(V=1, L=None):
    """S_r = members of NB at Chebyshev distance r, for r = 1..V (L defaults
    to cube_L(V), reading R17)."""
    nb = neighbourhood(cube_L(V) if L is None else L)
    return [[o for o in nb if max(abs(o[0]), abs(o[1]), abs(o[2])) == r]
            for r in range(1, V + 1)]


def shell_weights(V=1, h=1.0):
    """W_r = exp(-r/h) / sum_{s=1..V} exp(-s/h)   (Eq 10)."""
    e = np.array([math.exp(-r / h) for r in range(1, V + 1)])
    return e / e.sum()


def _overlap(n, d):
    """Index slices (centre i, neighbour k = i + d) along one axis of length n."""
    if d >= 0:
        return slice(0, max(n - d, 0)), slice(d, n)
    return slice(-d, n), slice(0, max(n + d, 0))


# --------------------------------------------------------------------------
# Eqs 5-8: neighbourhood terms H and F
# --------------------------------------------------------------------------
def neighbour_terms(x, U, V=1, h=1.0, L=None, return_aux=False):
    """H_ij (Eq 5, with g of Eq 6) and F_ij (Eq 7, with q^2 of Eq 8).

    Returns (H, F) of shape (c, nz, ny, nx); with ``return_aux`` also a dict
    of the per-shell denominators G (sum g) and Q (sum q^2) and the in-volume
    neighbour counts, for the tests.
    """
    x = np.asarray(x, dtype=np.float64)
    U = np.asarray(U, dtype=np.float64)
    c = U.shape[0]
    shape = x.shape
    W = shell_weights(V, h)
    H = np.zeros((c,) + shape)
    F = np.zeros((c,) + shape)
    wsum = np.zeros(shape)
    aux = {"G": [], "Q": [], "count": []}
    for r, offs in enumerate(shells(V, L)):
        numH = np.zeros((c,) + shape)
        numF = np.zeros((c,) + shape)
        sumU = np.zeros((c,) + shape)
        G = np.zeros(shape)
        Q = np.zeros(shape)
        cnt = np.zeros(shape)
        for dz, dy, dx in offs:
            iz, kz = _overlap(shape[0], dz)
            iy, ky = _overlap(shape[1], dy)
            ix, kx = _overlap(shape[2], dx)
            i_sl, k_sl = (iz, iy, ix), (kz, ky, kx)
            g = np.abs(x[i_sl] - x[k_sl])                  # Eq 6
            q2 = float(dx * dx + dy * dy + dz * dz)        # Eq 8 (reading R1)
            uk = U[(slice(None),) + k_sl]
            numH[(slice(None),) + i_sl] += uk * g
            numF[(slice(None),) + i_sl] += uk * uk * q2
            sumU[(slice(None),) + i_sl] += uk
            G[i_sl] += g
            Q[i_sl] += q2
            cnt[i_sl] += 1.0
        present = cnt > 0
        with np.errstate(divide="ignore", invalid="ignore"):
            Hr = np.where(G > 0, numH / G, sumU / cnt)     # Eq 5, reading R3
            Fr = numF / Q                                   # Eq 7
        H += np.where(present, W[r] * Hr, 0.0)
        F += np.where(present, W[r] * Fr, 0.0)
        wsum += np.where(present, W[r], 0.0)
        aux["G"].append(G)
        aux["Q"].append(Q)
        aux["count"].append(cnt)
    with np.errstate(divide="ignore", invalid="ignore"):
        H = np.where(wsum > 0, H / wsum, 0.0)
        F = np.where(wsum > 0, F / wsum, 0.0)
    if return_aux:
        return H, F, aux
    return H, F


# --------------------------------------------------------------------------
# Eq 4, Eq 2, Eq 1, Eq 3
# --------------------------------------------------------------------------
def modified_distance(x, C, H, F, lam, xi, dist_floor=1e-12):
    """d^2_ij = ||x_i - c_j||^2 (1 - lambda H_ij - xi F_ij)  (Eq 4, reading R2)."""
    x = np.asarray(x, dtype=np.float64)
    C = np.asarray(C, dtype=np.float64)
    diff2 = (x[None] - C.reshape((-1,) + (1,) * x.ndim)) ** 2
    factor = np.maximum(1.0 - lam * H - xi * F, 0.0)
    return np.maximum(diff2 * factor, dist_floor)


def membership(d2, m):
    """u_ij = 1 / sum_k (d_ij / d_ik)^(2/(m-1))  (Eq 2, written with d^2)."""
    e = 1.0 / (m - 1.0)
    total = np.zeros_like(d2)
    for k in range(d2.shape[0]):
        total += (d2 / d2[k][None]) ** e
    return 1.0 / total


def objective(U, d2, m):
    """J_m = sum_i sum_j u_ij^m d^2(x_i, c_j)  (Eq 1)."""
    return float(np.sum(U ** m * d2))


def centres(x, U, m):
    """c_j = sum_i u_ij^m x_i / sum_i u_ij^m  (Eq 3)."""
    w = U ** m
    axes = tuple(range(1, U.ndim))
    return np.sum(w * x[None], axis=axes) / np.sum(w, axis=axes)


# --------------------------------------------------------------------------
# The step function and its loop (Alg 1 step 4 / Alg 2 steps 6-10)
# --------------------------------------------------------------------------
def ifcm_iteration(x, U, C, lam, xi, m=2.0, V=1, h=1.0, dist_floor=1e-12, store=None):
    """One IFCM iteration t: (U^t, C^t) -> (U^{t+1}, C^{t+1}, J^t, delta^t).

    H and F come from U^t (R6); d^2 from C^t (Eq 4); U^{t+1} from Eq 2;
    J^t from Eq 1 with that d^2 (R7); C^{t+1} from Eq 3;
    delta^t = max_ij |u^{t+1}_ij - u^t_ij|.

    ``store`` (optional) models a storage format for the memberships: the
    returned U^{t+1} is store(U^{t+1}), and delta compares stored values.
    J^t and C^{t+1} are still taken from the unrounded U^{t+1}.
    """
    if lam == 0.0 and xi == 0.0:
        H = F = 0.0                       # Eq 4 reduces to plain FCM
    else:
        H, F = neighbour_terms(x, U, V=V, h=h)
    d2 = modified_distance(x, C, H, F, lam, xi, dist_floor)
    U1 = membership(d2, m)
    J = objective(U1, d2, m)
    C1 = centres(x, U1, m)
    if store is not None:
        U1 = store(U1)
    delta = float(np.max(np.abs(U1 - U)))
    return U1, C1, J, delta


def ifcm_fit(x, U0, C0, lam, xi, m=2.0, max_iter=50, eps=1e-5, V=1, h=1.0,
             dist_floor=1e-12, history=False, store=None):
    """Run IFCM from (U0, C0) until delta < eps or max_iter iterations (R5).

    Returns (U, C, J_last, iterations) and, with ``history``, the list of
    (J^t, delta^t) per iteration.  ``store`` models the storage format of the
    memberships (see ``ifcm_iteration``); the start U0 is stored first.
    """
    U = np.asarray(U0, dtype=np.float64)
    if store is not None:
        U = store(U)
    C = np.asarray(C0, dtype=np.float64)
    J = float("nan")
    hist = []
    it = 0
    for it in range(1, max_iter + 1):
        U, C, J, delta = ifcm_iteration(x, U, C, lam, xi, m, V, h, dist_floor, store)
        hist.append((J, delta))
        if delta < eps:
            break
    if history:
        return U, C, J, it, hist
    return U, C, J, it


def fcm_init(x, c, m=2.0, max_iter=300, eps=1e-5, dist_floor=1e-12):
    """Initial (U0, C0): plain FCM (lambda = xi = 0) from c_j = (j+1/2)/c,
    u_ij = 1/c  (Alg 1 step 2 / Alg 2 step 5, reading R10)."""
    x = np.asarray(x, dtype=np.float64)
    C = (np.arange(c, dtype=np.float64) + 0.5) / c
    U = np.full((c,) + x.shape, 1.0 / c)
    U, C, J, it = ifcm_fit(x, U, C, 0.0, 0.0, m, max_iter, eps,
                           dist_floor=dist_floor)
    return U, C, J, it


def labels(U):
    """Hard labels argmax_j u_ij, ties to the lowest j."""
    return np.argmax(U, axis=0)
