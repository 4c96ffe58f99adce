"""FP64 reverse-mode derivative of the IFCM objective with respect to
(lambda, xi) through K unrolled iterations (TEST INFRASTRUCTURE ONLY).

The differentiated function is L(lambda, xi) = J^{K-1}, the objective of the
last of K iterations from a fixed start (U^0, C^0) with no stop rule.  That is
the fitness of reading R5 with eps = 0 and max_iter = K.  Only the first
neighbourhood shell is supported (V = 1, W_1 = 1), as in the kernels.

Forward iteration t (the oracle's own ``ifcm.ifcm_iteration`` steps):
  H, F from U^t                                   (Eqs 5-8)
  D_ij = (x_i - c^t_j)^2,  f_ij = 1 - lambda H_ij - xi F_ij
  d2_ij = max(D_ij max(f_ij, 0), floor)           (Eq 4, reading R2)
  a_ij = d2_ij^(-p), p = 1/(m-1),  u_ij = a_ij / sum_k a_ik = U^{t+1}  (Eq 2)
  w = u^m,  J^t = sum w d2  (Eq 1),  c^{t+1}_j = sum_i w_ij x_i / S0_j,
  S0_j = sum_i w_ij  (Eq 3)

Reverse of iteration t, given the adjoints u_bar of U^{t+1} and c_bar of
C^{t+1}, and J_bar = 1 for t = K-1 (else 0):
  w_bar  = J_bar d2 + c_bar_j (x_i - c^{t+1}_j) / S0_j
  u_tot  = u_bar + m u^(m-1) w_bar
  d2_bar = J_bar w - p (u_tot - sum_k u_tot_k u_k) u / d2
  P_bar  = d2_bar where D max(f, 0) > floor (else 0)
  f_bar  = P_bar D where f > 0 (else 0)
  lambda_bar += sum -f_bar H,   xi_bar += sum -f_bar F
  c_bar^t_j   = sum_i -2 P_bar max(f, 0) (x_i - c^t_j)
  H_bar = -lambda f_bar,  F_bar = -xi f_bar
  u_bar^t_kj = sum over i with k in NB(i) of
       H_bar_ij g_ik / G_i   (or H_bar_ij / n_i where G_i = 0, reading R3)
     + F_bar_ij 2 u_kj q^2_ik / Q_i
The neighbourhood relation is symmetric (k in NB(i) iff i in NB(k), both
inside the volume), g_ik = g_ki and q^2_ik = q^2_ki, so the last sum is a
stencil over k's own neighbours.  Where D max(f,0) equals the floor exactly,
or f = 0 exactly, the one-sided derivative 0 is taken.
"""
import numpy as np

from . import ifcm as O


def _neighbour_terms_with_aux(x, U):
    """H, F (Eqs 5, 7 with V = 1) and the denominators G, Q and counts n."""
    H, F, aux = O.neighbour_terms(x, U, V=1, h=1.0, return_aux=True)
    return H, F, aux["G"][0], aux["Q"][0], aux["count"][0]


def _transpose_stencil(x, U, Hb_over, Fb_over, flat):
    """u_bar_kj = sum_{i: k in NB(i)} Hb_over_ij w_ik + 2 u_kj Fb_over_ij q^2_ik,
    with w_ik = g_ik, or 1 where i is flat (G_i = 0)."""
    shape = x.shape
    out = np.zeros_like(U)
    for dz, dy, dx in O.shells(1)[0]:
        iz, kz = O._overlap(shape[0], dz)
        iy, ky = O._overlap(shape[1], dy)
        ix, kx = O._overlap(shape[2], dx)
        i_sl, k_sl = (iz, iy, ix), (kz, ky, kx)
        g = np.abs(x[i_sl] - x[k_sl])
        wgt = np.where(flat[i_sl], 1.0, g)
        q2 = float(dx * dx + dy * dy + dz * dz)
        uk = U[(slice(None),) + k_sl]
        out[(slice(None),) + k_sl] += (Hb_over[(slice(None),) + i_sl] * wgt +
                                       2.0 * uk * Fb_over[(slice(None),) + i_sl] * q2)
    return out


def ifcm_grad(x, U0, C0, lam, xi, m=2.0, K=20, dist_floor=1e-12):
    """Return (J^{K-1}, dJ/dlambda, dJ/dxi) for K unrolled iterations."""
    x = np.asarray(x, dtype=np.float64)
    p = 1.0 / (m - 1.0)
    # forward, keeping every U^t and C^t (checkpoints)
    Us = [np.asarray(U0, dtype=np.float64)]
    Cs = [np.asarray(C0, dtype=np.float64)]
    J = None
    for _ in range(K):
        U1, C1, J, _ = O.ifcm_iteration(x, Us[-1], Cs[-1], lam, xi, m, 1, 1.0, dist_floor)
        Us.append(U1)
        Cs.append(C1)
    lam_bar = xi_bar = 0.0
    u_bar = np.zeros_like(Us[0])
    c_bar = np.zeros_like(Cs[0])
    bshape = (-1,) + (1,) * x.ndim
    for t in range(K - 1, -1, -1):
        U, C, u, C1 = Us[t], Cs[t], Us[t + 1], Cs[t + 1]
        J_bar = 1.0 if t == K - 1 else 0.0
        H, F, G, Q, n = _neighbour_terms_with_aux(x, U)
        D = (x[None] - C.reshape(bshape)) ** 2
        f = 1.0 - lam * H - xi * F
        fac = np.maximum(f, 0.0)
        P = D * fac
        d2 = np.maximum(P, dist_floor)
        w = u ** m
        S0 = np.sum(w, axis=tuple(range(1, w.ndim)))
        w_bar = J_bar * d2 + (c_bar / S0).reshape(bshape) * (x[None] - C1.reshape(bshape))
        u_tot = u_bar + m * u ** (m - 1.0) * w_bar
        d2_bar = J_bar * w - p * (u_tot - np.sum(u_tot * u, axis=0)[None]) * u / d2
        P_bar = np.where(P > dist_floor, d2_bar, 0.0)
        f_bar = np.where(f > 0.0, P_bar * D, 0.0)
        lam_bar += float(np.sum(-f_bar * H))
        xi_bar += float(np.sum(-f_bar * F))
        axes = tuple(range(1, x.ndim + 1))
        c_bar = np.sum(-2.0 * P_bar * fac * (x[None] - C.reshape(bshape)), axis=axes)
        flat = G == 0.0
        with np.errstate(divide="ignore", invalid="ignore"):
            Hb_over = np.where(flat[None], -lam * f_bar / n[None], -lam * f_bar / G[None])
            Fb_over = np.where(Q[None] > 0, -xi * f_bar / Q[None], 0.0)
        Hb_over = np.where(n[None] > 0, Hb_over, 0.0)
        u_bar = _transpose_stencil(x, U, Hb_over, Fb_over, flat)
    return J, lam_bar, xi_bar
