"""The identity behind the engine's deferred NLMS step, checked in FP64 on the
oracle's own recursion (CPU, no engine).

The engine does not apply block n's step to partitions j >= 1 before block
n's prediction; it forms the same prediction as

    C_n = sum_l F_n[0] U_n + sum_l sum_{j>=1} F_{n-2}[j] U_{n-j} + G_n A1_n + G_{n-1} A2_n,
    A1_n = sum_l sum_{j>=1} conj(U_{n-1-j}) U_{n-j},  A2_n = sum_l sum_{j>=1} conj(U_{n-2-j}) U_{n-j},

with U_m the loudspeaker spectra of block m, F_m the sub-filter spectra after
block m's step and G_m the step-scaled error spectrum (the factor of conj(U)
in the update).  This holds because the update is linear in F.  The test runs
``NlmsCanceller`` (the literal recursion) and compares its prediction spectra
with the right-hand side, bin by bin, to FP64 rounding; a planted mistake in
the right-hand side (a lag off by one) must fail.
"""

import numpy as np

from oracle.nlms_oracle import NlmsCanceller


def run_recursion(P=2, L=3, B=16, n_t=70, nb=14, mu=0.4, lam=0.8, delta=1e-2, seed=3):
    rng = np.random.default_rng(seed)
    can = NlmsCanceller(rng.standard_normal((P, L, n_t)) * 0.3, B, mu, lam, delta)
    K = can.K
    U = {}  # block -> [L][B+1] loudspeaker spectra
    F = {-1: can.W.copy()}  # block -> spectra after that block's step
    G = {}  # block -> [P][B+1] step-scaled error spectra
    C = {}  # block -> [P][B+1] prediction spectra of the literal recursion
    for n in range(nb):
        e_n = rng.standard_normal((P, B)) * 0.1
        # the step as the oracle takes it: power over the newest entry, then E * mu / (K pow + delta)
        inst = np.sum(np.abs(can.fdl[0]) ** 2, axis=0)
        pow_n = can.lam * can.power + (1.0 - can.lam) * inst
        G[n] = can.error_spectrum(e_n) * (can.mu / (K * pow_n + can.delta))[None, :]
        can.adapt(e_n)
        F[n] = can.W.copy()
        l_n = rng.standard_normal((L, B)) * 0.2
        can.predict(l_n)
        U[n] = can.fdl[0].copy()
        C[n] = np.einsum("pljk,jlk->pk", can.W, can.fdl)
    return can, K, U, F, G, C


def entry(U, m, L, B):
    return U.get(m, np.zeros((L, B + 1), dtype=np.complex128))


def deferred(U, F, G, K, n, L, B, lag2=2):
    head = np.einsum("plk,lk->pk", F[n][:, :, 0, :], U[n])
    tail = sum(np.einsum("plk,lk->pk", F[n - 2][:, :, j, :], entry(U, n - j, L, B)) for j in range(1, K))
    A1 = sum(np.sum(np.conj(entry(U, n - 1 - j, L, B)) * entry(U, n - j, L, B), axis=0) for j in range(1, K))
    A2 = sum(np.sum(np.conj(entry(U, n - lag2 - j, L, B)) * entry(U, n - j, L, B), axis=0) for j in range(1, K))
    return head + tail + G[n] * A1[None, :] + G[n - 1] * A2[None, :]


def test_deferred_prediction_equals_the_literal_recursion():
    P, L, B = 2, 3, 16
    can, K, U, F, G, C = run_recursion(P=P, L=L, B=B)
    assert K >= 4
    F[-2] = F[-1]
    G[-1] = np.zeros_like(G[0])
    for n in range(len(C)):
        rhs = deferred(U, F, G, K, n, L, B)
        err = np.max(np.abs(rhs - C[n])) / np.max(np.abs(C[n]))
        assert err < 1e-12, (n, err)


def test_a_wrong_lag_fails():
    P, L, B = 2, 3, 16
    can, K, U, F, G, C = run_recursion(P=P, L=L, B=B)
    F[-2] = F[-1]
    G[-1] = np.zeros_like(G[0])
    worst = max(np.max(np.abs(deferred(U, F, G, K, n, L, B, lag2=3) - C[n])) / np.max(np.abs(C[n]))
                for n in range(2, len(C)))
    assert worst > 1e-3
