"""Plain numpy FP64 restatement of the analysis of a simulation history (test infrastructure only).

Follows the quantities the paper extracts from the stored energy and magnetization (Sec. II:
thermal averages and correlation times from the history; Sec. IV.A thermal averages M, chi;
Sec. IV.B the finite-size-scaling cumulants; Sec. IV.E single and multiple histogram
methods), with the textbook definitions written out:

  per series (one temperature/field step of one instance, records after a cut):
    e  = <E>/N                      m  = <|M|>/N
    c  = (<E^2> - <E>^2) / (N T^2)  chi = (<M^2> - <|M|>^2) / (N T)      (k_B = 1)
    u4 = 1 - <M^4> / (3 <M^2>^2)                                         (Binder cumulant)
    v1 = <E> - <|M| E> / <|M|>      v2 = <E> - <M^2 E> / <M^2>
         (v_j = d ln<|M|^j> / d beta, Ferrenberg & Landau, PRB 44, 5081 (1991))
    errors: e, m from n_bins equal bins (standard error of the bin means); c, chi, u4 by
            the jackknife over the same bins
    tau_e, tau_m: integrated autocorrelation times of E and |M| (MCS), Sokal's automatic
            window: tau(W) = 1/2 + sum_{t=1..W} rho(t), the smallest W >= 6 tau(W), at most n/2
  reweighting (Ferrenberg & Swendsen, PRL 61, 2635 (1988); PRL 63, 1195 (1989)):
    K runs at beta_k with n samples each; ln Z_k = g_k solves
      g_k = ln sum_i exp(-beta_k E_i - D_i),  D_i = ln sum_j n exp(-beta_j E_i - g_j),
    iterated from g = 0 with the gauge g_0 = 0; then
      <O>_beta = sum_i O_i exp(-beta E_i - D_i) / sum_i exp(-beta E_i - D_i).
    K = 1 is the single-histogram method.

Binning: b = n // n_bins samples per bin over the first b * n_bins samples after the cut.
"""

from __future__ import annotations

import numpy as np

FIELDS = ("e", "e_err", "m", "m_err", "c", "c_err", "chi", "chi_err", "u4", "u4_err", "v1", "v2", "tau_e",
          "tau_m", "n", "bins")


def tau_int(x, c: float = 6.0) -> float:
    """Integrated autocorrelation time with Sokal's automatic window (c = 6)."""
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[0]
    d = x - x.mean()
    c0 = np.dot(d, d) / n
    if c0 == 0.0:
        return 0.5
    tau = 0.5
    for t in range(1, n // 2 + 1):
        rho = (np.dot(d[:-t], d[t:]) / (n - t)) / c0
        tau += rho
        if t >= c * tau:
            break
    return float(tau)


def _estimates(E, A, M2, N, T):
    """(c, chi, u4) from samples of E, |M| and M^2."""
    c = np.var(E) / (N * T * T)
    chi = np.var(A) / (N * T)
    u4 = 1.0 - np.mean(M2 * M2) / (3.0 * np.mean(M2) ** 2)
    return np.array([c, chi, u4])


def thermal_averages(series, cut: int, n_bins: int, T: float, N: float) -> dict:
    """series: [len, 4] (E, Mx, My, Mz) after every MCS of one step. Returns a dict of FIELDS."""
    h = np.asarray(series, dtype=np.float64)[cut:]
    n = h.shape[0]
    E = h[:, 0]
    M2 = (h[:, 1:] ** 2).sum(axis=1)
    A = np.sqrt(M2)
    out = dict(e=E.mean() / N, m=A.mean() / N)
    c, chi, u4 = _estimates(E, A, M2, N, T)
    out.update(c=c, chi=chi, u4=u4)
    out["v1"] = E.mean() - np.mean(A * E) / A.mean()
    out["v2"] = E.mean() - np.mean(M2 * E) / M2.mean()
    b = n // n_bins
    used = slice(0, b * n_bins)
    Eb = E[used].reshape(n_bins, b)
    Ab = A[used].reshape(n_bins, b)
    M2b = M2[used].reshape(n_bins, b)
    out["e_err"] = Eb.mean(axis=1).std(ddof=1) / np.sqrt(n_bins) / N
    out["m_err"] = Ab.mean(axis=1).std(ddof=1) / np.sqrt(n_bins) / N
    jk = np.array([_estimates(np.delete(Eb, k, axis=0).ravel(), np.delete(Ab, k, axis=0).ravel(),
                              np.delete(M2b, k, axis=0).ravel(), N, T) for k in range(n_bins)])
    err = np.sqrt((n_bins - 1) / n_bins * ((jk - jk.mean(axis=0)) ** 2).sum(axis=0))
    out["c_err"], out["chi_err"], out["u4_err"] = err
    out["tau_e"] = tau_int(E)
    out["tau_m"] = tau_int(A)
    out["n"] = float(n)
    out["bins"] = float(n_bins)
    return out


def reweight(E, O, betas_k, betas_out, max_iter: int = 10000, tol: float = 1e-12):
    """E: [K, n] energies of K runs at betas_k; O: [K, n, n_obs] observables. Returns
    (<O> at betas_out [n_out, n_obs], g [K] = ln Z_k - ln Z_0, iterations used)."""
    E = np.asarray(E, dtype=np.float64)
    K, n = E.shape
    O = np.asarray(O, dtype=np.float64).reshape(K * n, -1)
    bk = np.asarray(betas_k, dtype=np.float64)
    Ei = E.reshape(-1)
    g = np.zeros(K)
    it = 0
    for it in range(1, max_iter + 1):
        D = np.logaddexp.reduce(np.log(n) - np.outer(Ei, bk) - g[None, :], axis=1)
        g_new = np.logaddexp.reduce(-np.outer(bk, Ei) - D[None, :], axis=1)
        g_new -= g_new[0]
        done = np.max(np.abs(g_new - g)) < tol
        g = g_new
        if done:
            break
    D = np.logaddexp.reduce(np.log(n) - np.outer(Ei, bk) - g[None, :], axis=1)
    out = []
    for b in np.asarray(betas_out, dtype=np.float64):
        lw = -b * Ei - D
        w = np.exp(lw - lw.max())
        out.append((w[:, None] * O).sum(axis=0) / w.sum())
    return np.array(out), g, it
