"""Growth series and steady-state statistics (Kelling & Odor, Secs. III and IV).

* The growth run: W^2 at log-spaced sample times (the paper's Eq. (8)
  recursion read as n log-spaced times over T), the growth exponent beta as
  the slope of (1/2) ln(W^2 - W^2(0)) against ln t (Sec. III), and its local
  slopes beta_eff (Eq. (11)).

* The distribution of the squared width W^2 in the steady state: its
  cumulants kappa_1..kappa_4, written through the raw moments
  nu_n = <(W^2)^n> (Sec. IV, the cumulant-moment relations), and the scaled
  distribution Psi_L(x) = <W^2> P_L(W^2 / <W^2>) (Sec. IV).
* The effective roughness exponent alpha_eff(L) (Sec. III, Eq. (13)) and the
  finite-size-scaling fit alpha_eff(L) = alpha + a1 w1 L^(-w1) (Eq. (14),
  correction exponent read with a minus sign so that it vanishes as L grows).
* The power spectrum S(k) on the axes (Sec. III, Eqs. (15)-(16)) averaged
  over replicas and sampling times.

Samples come from batched replicas (okz_batch_*): every replica is run to the
steady state and then sampled every `every` sweeps; each W^2 sample is exact
(Eq. (4)), each spectrum is computed on the device (okz_psd).
"""
import math

import numpy as np

import paper_1110_6745_gb300 as okz


def w2_cumulants(samples):
    """kappa_1..kappa_4 of the samples from their raw moments nu_n:
    kappa_1 = nu_1, kappa_2 = nu_2 - nu_1^2,
    kappa_3 = nu_3 - 3 nu_1 nu_2 + 2 nu_1^3,
    kappa_4 = nu_4 - 4 nu_3 nu_1 - 3 nu_2^2 + 12 nu_1^2 nu_2 - 6 nu_1^4,
    evaluated in extended precision."""
    x = np.asarray(samples, dtype=np.longdouble).ravel()
    nu = [np.mean(x ** n) for n in range(1, 5)]
    n1, n2, n3, n4 = nu
    k1 = n1
    k2 = n2 - n1 * n1
    k3 = n3 - 3 * n1 * n2 + 2 * n1 ** 3
    k4 = n4 - 4 * n3 * n1 - 3 * n2 * n2 + 12 * n1 * n1 * n2 - 6 * n1 ** 4
    return [float(k) for k in (k1, k2, k3, k4)]


def psi(samples, bins=50):
    """Psi_L(x) = <W^2> P_L(W^2 / <W^2>): a normalised histogram of
    x = W^2 / <W^2>. Returns (bin centres, density)."""
    w = np.asarray(samples, dtype=np.float64).ravel()
    x = w / w.mean()
    dens, edges = np.histogram(x, bins=bins, density=True)
    return 0.5 * (edges[1:] + edges[:-1]), dens


def steady_state_w2(L, replicas, burnin, nsamples, every, p=1.0, q=0.0, seed0=0, tune=False):
    """W^2 samples (replicas x nsamples) of `replicas` independent lattices of
    size L (seeds seed0 + r), each run `burnin` sweeps from the striped start
    and then sampled every `every` sweeps. With `tune` the batch's launch shape
    is autotuned first (results do not depend on it)."""
    with okz.Batch([L] * replicas, [p] * replicas, [q] * replicas,
                   [seed0 + r for r in range(replicas)]) as b:
        if tune:
            b.autotune(probe_sweeps=2)
        _advance(b, replicas, burnin)
        out = np.empty((replicas, nsamples))
        for k in range(nsamples):
            _advance(b, replicas, every)
            W2, _, _ = b.stats()
            out[:, k] = W2
    return out


def _advance(b, replicas, sweeps, per_launch=1 << 16):
    """All replicas of batch b forward by `sweeps`, at most `per_launch` sweeps
    per batched launch (keeps single launches short)."""
    while sweeps > 0:
        n = min(sweeps, per_launch)
        b.run([n] * replicas)
        sweeps -= n


def alpha_eff(Ls, w2_means):
    """alpha_eff(L) = [ln W(L) - ln W(L/2)] / ln 2 (Eq. (13)) with W = sqrt(<W^2>),
    for every L in Ls whose half is also in Ls. Returns (L values, alpha_eff)."""
    w = dict(zip((int(l) for l in Ls), (float(v) for v in w2_means)))
    out_L, out_a = [], []
    for L in sorted(w):
        if L // 2 in w and L % 2 == 0:
            out_L.append(L)
            out_a.append(0.5 * (np.log(w[L]) - np.log(w[L // 2])) / np.log(2.0))
    return np.array(out_L), np.array(out_a)


def fit_alpha(Ls, a_eff, omega):
    """Least-squares fit of alpha_eff(L) = alpha + c L^(-omega) (Eq. (14),
    c = a1 omega) at a fixed correction exponent omega. Returns (alpha, c)."""
    Ls = np.asarray(Ls, dtype=np.float64)
    A = np.stack([np.ones_like(Ls), Ls ** (-float(omega))], axis=1)
    (alpha, c), *_ = np.linalg.lstsq(A, np.asarray(a_eff, dtype=np.float64), rcond=None)
    return float(alpha), float(c)


def alpha_fss(samples_by_L, omega=1.16, blocks=32):
    """Finite-size scaling of the steady-state width (Sec. III, Eqs. (13),
    (14)) with errors: alpha_eff(L) from the replica-and-sample means of W^2
    at L and L/2, and the fit alpha_eff(L) = alpha + c L^(-omega) at the fixed
    correction exponent omega. samples_by_L maps L to a (replicas x samples)
    array of W^2. Errors by delete-one-block jackknife: every L's replicas are
    split into `blocks` groups and block b is left out at every L at once.
    Returns a dict: L, alpha_eff, alpha_eff_err, alpha, alpha_err, c, c_err."""
    Ls = sorted(int(L) for L in samples_by_L)
    arrs = {L: np.asarray(samples_by_L[L], dtype=np.float64) for L in Ls}

    def estimate(drop=None):
        means = []
        for L in Ls:
            a = arrs[L]
            if drop is not None:
                idx = np.array_split(np.arange(a.shape[0]), blocks)[drop]
                a = np.delete(a, idx, axis=0)
            means.append(a.mean())
        Le, ae = alpha_eff(Ls, means)
        if len(Le) >= 2:
            al, c = fit_alpha(Le, ae, omega)
        else:
            al, c = float("nan"), float("nan")
        return Le, ae, al, c

    Le, ae, al, c = estimate()
    jk = [estimate(b) for b in range(blocks)]
    f = (blocks - 1) / blocks
    ae_j = np.array([j[1] for j in jk])
    al_j = np.array([j[2] for j in jk])
    c_j = np.array([j[3] for j in jk])
    err = lambda v: float(np.sqrt(f * np.sum((v - v.mean(axis=0)) ** 2, axis=0))) \
        if np.ndim(v) == 1 else np.sqrt(f * np.sum((v - v.mean(axis=0)) ** 2, axis=0))
    return {"L": [int(x) for x in Le], "alpha_eff": [float(x) for x in ae],
            "alpha_eff_err": [float(x) for x in err(ae_j)], "alpha": float(al),
            "alpha_err": err(al_j), "c": float(c), "c_err": err(c_j), "omega": float(omega)}


def steady_state_psd(L, replicas, burnin, nsamples, every, p=1.0, q=0.0, seed0=0):
    """The axis spectrum S[k] (okz_psd) averaged over `replicas` lattices of
    size L (seeds seed0 + r) and `nsamples` times `every` sweeps apart after
    `burnin` sweeps. The replicas run batched; each sample's state is moved
    into one simulation (okz_restore) whose spectrum is taken on the device."""
    acc = np.zeros(int(L))
    with okz.Batch([L] * replicas, [p] * replicas, [q] * replicas,
                   [seed0 + r for r in range(replicas)]) as b, \
            okz.Simulation(L, p, q, seed=seed0, kernel=okz.OKZ_KERNEL_PARITY_PLAIN) as sim:
        _advance(b, replicas, burnin)
        for _ in range(nsamples):
            _advance(b, replicas, every)
            for r in range(replicas):
                planes, H0, t = b.state(r)
                sim.restore(planes, H0, t)
                acc += sim.psd()
    return acc / (replicas * nsamples)


def spectrum_slope(S, kmin, kmax):
    """Least-squares slope of ln S[k] against ln k over kmin <= k <= kmax
    (indices, k standing for 2 pi k / L); S ~ k^(-2-2 alpha) in the steady
    state (Sec. III)."""
    k = np.arange(len(S))
    m = (k >= kmin) & (k <= kmax)
    return float(np.polyfit(np.log(k[m]), np.log(np.asarray(S)[m]), 1)[0])


def sample_times(T, n):
    """[0] + n log-spaced sweep counts over T: t_j = max(round(T^(j/(n-1))),
    t_(j-1) + 1), j = 0 .. n-1, rounding halves away from zero (so t_(n-1) = T).
    Requires 2 <= n <= T."""
    T, n = int(T), int(n)
    if n < 2 or n > T:
        raise ValueError("need 2 <= n <= T")
    out, prev = [0], 0
    for j in range(n):
        v = int(math.floor(math.pow(float(T), j / (n - 1)) + 0.5))
        v = max(v, prev + 1)
        out.append(v)
        prev = v
    if out[-1] != T:
        raise ValueError("the schedule does not end at T")
    return out


def growth_series(L, T, n, p=1.0, q=0.0, seed=0, s_sel=0.5, kernel=None):
    """A growth run from the striped start: one simulation swept to every
    sample time of sample_times(T, n); returns records (t, H0, S1, S2, W2)
    with the exact sums of h and h^2 (Eq. (4))."""
    kw = {} if kernel is None else {"kernel": kernel}
    with okz.Simulation(L, p, q, seed=seed, s_sel=s_sel, **kw) as sim:
        # sweeps and exact sums queued on the device, one synchronisation
        return [tuple(r) for r in sim.growth_series(sample_times(T, n))]


def beta_fit(t, w2, tmin, tmax, w2_0=0.25):
    """Least-squares slope of (1/2) ln(W^2 - w2_0) against ln t over
    tmin <= t <= tmax (Sec. III: the constant W^2(0) = 1/4 of the striped start
    is subtracted first)."""
    t = np.asarray(t, dtype=np.float64)
    w2 = np.asarray(w2, dtype=np.float64)
    m = (t >= tmin) & (t <= tmax)
    return float(np.polyfit(np.log(t[m]), 0.5 * np.log(w2[m] - w2_0), 1)[0])


def beta_eff(t, w2, ratio=2.0, w2_0=0.25):
    """Local slopes of Eq. (11): beta_eff(t) = [ln W(t) - ln W(t')] /
    [ln t - ln t'] with W^2 - w2_0 for W^2 and t' the latest sample time
    <= t / ratio. Returns (t values, beta_eff) for every t that has such a t'
    > 0."""
    ts = [float(x) for x in t]
    w = [float(x) - w2_0 for x in w2]
    out_t, out_b = [], []
    for i, ti in enumerate(ts):
        prev = [j for j in range(i) if 0 < ts[j] <= ti / ratio]
        if not prev:
            continue
        j = prev[-1]
        out_t.append(ti)
        out_b.append(0.5 * (math.log(w[i]) - math.log(w[j])) / (math.log(ti) - math.log(ts[j])))
    return np.array(out_t), np.array(out_b)
