"""Observation merging in the pseudo-inverse preconditioner (oracle, test-only).

App. A.3: if two bands have identical normalised inverse noise N~^-1 and proportional rows
of U (U_2 = gamma U_1: the same beam, frequency and SEDs, as for detector splits of one
channel), their share of U^T T U is

    U_1^T N~^-1 U_1 + U_2^T N~^-1 U_2 = (1 + gamma^2) U_1^T N~^-1 U_1,

so one row sqrt(1 + gamma^2) U_1 with that N~ replaces both, and M_PI needs one SHT pair
for the two.  (The paper prints the factor as (gamma + 1)^1/2; the algebra gives
(1 + gamma^2)^1/2, which is used.)  For bands that are only similar the paper asks for
compromise beams, noise and mixing; the oracle takes, for a group G of bands on one grid:

* row:   per l the best rank-one fit of sum_{nu in G} U_nu^T U_nu (Eckart-Young):
         u_G = sqrt(lambda_max) v_max, the sign making the largest entry of v positive;
         for proportional rows this is the exact merge above;
* noise: the co-added inverse noise tau_G = sum_{nu in G} tau_nu, alpha_G from
         Eq. optimal-alpha, T_G^+ = alpha_G^2 Y^T W N_G W Y with N_G = diag(1 / tau_G);
         for exact splits (tau_nu = c_nu tau_1) T_G^+ = T_1^+.

The merged preconditioner is M = U'^+ T'^+ (U'^+)^T with U' = [u_G rows ; S^-1/2 rows].

Parity: pinned (tests/test_oracle_merge.py) -- for exact splits the merged U' has the same
U'^T U' as U (the identity of App. A.3) and the merged M equals M_PI, in the flat case
both equal A^-1 (one PCG iteration); the rank-one row against the leading singular pair of
the stacked rows (numpy SVD); the printed (gamma + 1)^1/2 factor fails the identity.
"""
import numpy as np

from . import alm as _alm
from . import precond as _pc
from . import sht as _sht


def check_groups(model, groups):
    seen = sorted(nu for G in groups for nu in G)
    if seen != list(range(model.nobs)) or any(len(G) == 0 for G in groups):
        raise ValueError("groups must partition the bands")
    for G in groups:
        if any(model.grids[nu] is not model.grids[G[0]] for nu in G):
            raise ValueError("bands of a group must share one grid")


def rank_one_row(R):
    """Row u with u^T u the best rank-one fit of R^T R (R: member rows, [|G|, Ncomp])."""
    S = R.T @ R
    if not np.any(S):
        return np.zeros(R.shape[1])
    w, V = np.linalg.eigh(S)
    v = V[:, -1]
    if v[np.argmax(np.abs(v))] < 0:
        v = -v
    return np.sqrt(max(w[-1], 0.0)) * v


def merged_U_blocks(model, groups):
    """U' per l, [Lmax+1, ngroups+Ncomp, Ncomp]."""
    check_groups(model, groups)
    U = _pc.U_blocks(model)
    ng, nobs = len(groups), model.nobs
    Um = np.zeros((U.shape[0], ng + model.ncomp, model.ncomp))
    for l in range(U.shape[0]):
        for g, G in enumerate(groups):
            Um[l, g] = rank_one_row(U[l, G, :])
    Um[:, ng:] = U[:, nobs:]
    return Um


def merged_tau(model, groups):
    return [np.sum([model.tau[nu] for nu in G], axis=0) for G in groups]


def apply_merged_precond(model, groups, r, Up=None):
    """z = U'^+ T'^+ (U'^+)^T r."""
    if Up is None:
        Up = _pc.pinv_blocks(merged_U_blocks(model, groups))
    taus = merged_tau(model, groups)
    Lw = Up.shape[0] - 1
    R = _pc._stack_to_3d(model, np.asarray(r, dtype=np.float64), Lw)
    t = np.einsum("lkj,lmk->lmj", Up, R)
    for g, G in enumerate(groups):
        grid = model.grids[G[0]]
        Ln = model.lmax_band[G[0]]
        w = grid.pixel_weights()
        a = _pc.optimal_alpha(taus[g], w)
        f = _sht.synthesis(grid, Ln, _alm.from_2d(t[..., g], Ln))
        f = f * (a * a * w * w / taus[g])
        t[..., g] = _alm.to_2d(_sht.adjoint(grid, Ln, f), Ln, Lw)
    Z = np.einsum("lkj,lmj->lmk", Up, t)
    return _pc._3d_to_stack(model, Z)
