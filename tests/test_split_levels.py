"""The reading behind r_hat > 32 on the GPU: a region's knots may enter the
prior in two steps (Sec. 1.1 recursion).  Projecting the remainder covariance
on the first half Q1 of a region's knots, then the new remainder on the second
half Q2 (same region), removes exactly C(., Q)C(Q, Q)^{-1}C(Q, .) for
Q = Q1 u Q2: the second step's matrix is the Schur complement of C(Q1, Q1) in
C(Q, Q).  So Sigma_MRA and the likelihood are unchanged.  Checked here on the
dense form of the oracle's model (brute force on small trees), and the check
is shown to catch a plausible mistake: projecting the second half on the
covariance before the first half was removed."""
import numpy as np
import pytest

from oracle import dense
from paper_1905_00141_gb300 import synth


def _sigma_two_step(part, sigma2, beta, wrong_second_step=False):
    """Dense Sigma_MRA with every non-leaf level entered as two projections:
    the first ceil(r_hat/2) knots of each region, then the rest."""
    _, info = dense.sigma_mra(part, sigma2, beta, return_all=True)
    X, Y, reg, knot_ids, n = info["X"], info["Y"], info["reg"], info["knot_ids"], info["n_obs"]
    M = part.M
    D = np.sqrt((X[:, None] - X[None, :]) ** 2 + (Y[:, None] - Y[None, :]) ** 2)
    Cm = sigma2 * np.exp(-D / beta)
    Sig = np.zeros_like(Cm)
    for m in range(M - 1):
        C_level = Cm.copy()
        for half in (0, 1):
            proj = np.zeros_like(Cm)
            src = C_level if (wrong_second_step and half == 1) else Cm
            for k, q in enumerate(knot_ids[m]):
                h = (len(q) + 1) // 2
                qh = q[:h] if half == 0 else q[h:]
                members = np.nonzero(reg[m] == k)[0]
                if len(members) == 0 or len(qh) == 0:
                    continue
                CaQ = src[np.ix_(members, qh)]
                proj[np.ix_(members, members)] = CaQ @ np.linalg.solve(src[np.ix_(qh, qh)], CaQ.T)
            Sig += proj
            nxt = reg[m] if half == 0 else reg[m + 1]
            Cm = np.where(nxt[:, None] == nxt[None, :], Cm - proj, 0.0)
    Sig += np.where(reg[M - 1][:, None] == reg[M - 1][None, :], Cm, 0.0)
    return Sig[:n, :n]


@pytest.mark.parametrize("n,M,J,r,seed", [(220, 3, 2, 49, 1), (200, 2, 4, 49, 2), (240, 4, 2, 36, 3),
                                          (180, 3, 4, 64, 4)])
def test_two_step_knots_give_the_same_sigma(n, M, J, r, seed):
    x, y, z = synth.uniform(n, seed)
    part = dense.Partition(x, y, z, M, J, r)
    for s2, beta in [(1.0, 0.1), (2.0, 0.3), (0.6, 0.03)]:
        S = dense.sigma_mra(part, s2, beta)
        S2 = _sigma_two_step(part, s2, beta)
        assert np.max(np.abs(S2 - S)) <= 1e-9 * s2
        tau2 = 0.05
        l1 = dense.gauss_loglik(S + tau2 * np.eye(len(S)), part.z)
        l2 = dense.gauss_loglik(S2 + tau2 * np.eye(len(S)), part.z)
        assert abs(l1 - l2) <= 1e-9 * abs(l1)


def test_two_step_check_catches_a_wrong_second_step():
    x, y, z = synth.uniform(220, 1)
    part = dense.Partition(x, y, z, 3, 2, 49)
    S = dense.sigma_mra(part, 1.0, 0.1)
    bad = _sigma_two_step(part, 1.0, 0.1, wrong_second_step=True)
    assert np.max(np.abs(bad - S)) > 1e-3
