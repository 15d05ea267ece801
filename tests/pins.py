"""Checks that pin the FP64 oracle to facts fixed by the paper and by
mathematics, independently of the oracle's own code.

Each ``pin_*`` function raises AssertionError when the oracle currently
loaded by ``oracle`` disagrees.  The oracle tests call them one by one; the
mutation test calls all of them against deliberately broken builds of the
oracle source and requires each planted mistake to be caught by at least one.

References are to the sections and equations of arXiv:2208.01525:
Sec. II (model, Eqs. 1-11), Sec. III (PRS scaling Eq. 12, continuum
equations Eqs. 13-16, leapfrog Eqs. 17-26, cooling Eqs. 27-30),
Sec. III.A (diagnostics Eqs. 31-37), Sec. III.B (cell overlap), Sec. IV
(Gauss law check, criticality lambda = 2 e^2).
"""
from __future__ import annotations

import math

import numpy as np

import oracle as O
import synth

TWO_PI = 2.0 * math.pi


# ---- independent helpers (written from the paper, not from the oracle) ----

class Expansion:
    """a(eta)/a(eta_ref) and a'/a for a ~ t^m in cosmic time, built without the
    closed-form exponent m / (1 - m) the oracle uses: with a = (t / t_ref)^m
    and d eta = dt / a, a obeys da/d eta = (m / t_ref) a^{2 - 1/m}, where
    t_ref = eta_ref / int_0^1 u^{-m} du (the integral done by scipy.quad);
    the ODE is integrated from a(eta_ref) = 1 with dense output."""

    def __init__(self, m, eta_ref, eta_lo, eta_hi):
        self.m = m
        if m == 0.0:
            return
        from scipy.integrate import quad, solve_ivp
        t_ref = eta_ref / quad(lambda u: u ** (-m), 0.0, 1.0)[0]
        self.k = m / t_ref
        rhs = lambda e, y: [self.k * y[0] ** (2.0 - 1.0 / m)]  # noqa: E731
        lo, hi = min(eta_lo, eta_ref), max(eta_hi, eta_ref)
        up = solve_ivp(rhs, (eta_ref, hi + 1e-9), [1.0], rtol=1e-12, atol=1e-14, dense_output=True)
        dn = solve_ivp(rhs, (eta_ref, lo - 1e-9), [1.0], rtol=1e-12, atol=1e-14, dense_output=True)
        self._up, self._dn, self._ref = up.sol, dn.sol, eta_ref

    def a(self, eta):
        if self.m == 0.0:
            return 1.0
        return float((self._up if eta >= self._ref else self._dn)(eta)[0])

    def hubble(self, eta):
        """a'/a with respect to conformal time."""
        if self.m == 0.0:
            return 0.0
        return self.k * self.a(eta) ** (1.0 - 1.0 / self.m)


def step_coefficients(p: O.Params, n: int):
    """(a_n, c_n, delta_n, omega_n) from Eqs. 12, 19 and 22, with a and
    d ln a / d ln eta = eta a'/a from Expansion."""
    eta = p.eta0 + n * p.deta
    ex = Expansion(p.m, p.eta_ref, eta, eta)
    a = ex.a(eta)
    delta = 0.5 * p.alpha * eta * ex.hubble(eta) * p.deta / eta
    return a, a ** (2 * p.beta), delta, delta * (1.0 - p.beta)


def cplx(st, s):
    return st[2 * s] + 1j * st[2 * s + 1]


def mom(st, s):
    return st[10 + 2 * s] + 1j * st[11 + 2 * s]


def roll(a, shift, axis_dir):
    """a(x + shift * e_dir) for dir 0 = x, 1 = y, 2 = z on arrays (nz, ny, nx)."""
    return np.roll(a, -shift, axis=2 - axis_dir)


def divergence_E(st, s, dx, base=14):
    """sum_i (E_i(x) - E_i(x - i)) / dx for the electric field of sector s."""
    return sum((st[base + 3 * s + i] - roll(st[base + 3 * s + i], -1, i)) / dx for i in range(3))


def gauge_transform(p: O.Params, st, lam_site):
    """phi -> e^{i Lambda} phi, pi -> e^{i Lambda} pi,
    A_i -> A_i + (Lambda(x+i) - Lambda(x)) / dx, E unchanged (both sectors)."""
    out = st.copy()
    g = np.exp(1j * lam_site)
    for s in range(2):
        f = cplx(st, s) * g
        m = mom(st, s) * g
        out[2 * s], out[2 * s + 1] = f.real, f.imag
        out[10 + 2 * s], out[11 + 2 * s] = m.real, m.imag
        for i in range(3):
            out[4 + 3 * s + i] = st[4 + 3 * s + i] + (roll(lam_site, 1, i) - lam_site) / p.dx
    return out


def swap_sectors(st):
    out = st.copy()
    out[0:2], out[2:4] = st[2:4], st[0:2]
    out[4:7], out[7:10] = st[7:10], st[4:7]
    out[10:12], out[12:14] = st[12:14], st[10:12]
    out[14:17], out[17:20] = st[17:20], st[14:17]
    return out


def bruteforce_windings(p: O.Params, st):
    """Plaquette windings from per-site phases: every edge difference
    alpha(x+i) - alpha(x) - dx A_i(x) is brought into (-pi, pi] by adding or
    subtracting 2 pi in a loop (long double), and the oriented sum of
    (reduced difference + dx A) around each plaquette is divided by 2 pi."""
    ld = np.longdouble
    pi_l = ld(np.pi)
    W = np.zeros((2, 3) + p.shape, dtype=np.int64)
    planes = ((0, 1), (0, 2), (1, 2))
    for s in range(2):
        alpha = np.angle(cplx(st, s)).astype(ld)
        theta = [st[4 + 3 * s + i].astype(ld) * ld(p.dx) for i in range(3)]

        def edge(i, shift_dirs):
            a0 = alpha
            th = theta[i]
            for d in shift_dirs:
                a0 = roll(a0, 1, d)
                th = roll(th, 1, d)
            a1 = roll(a0, 1, i)
            d = a1 - a0 - th
            d = d.copy()
            for _ in range(64):
                hi = d > pi_l
                lo = d <= -pi_l
                if not (hi.any() or lo.any()):
                    break
                d[hi] -= 2 * pi_l
                d[lo] += 2 * pi_l
            return d + th

        for k, (i, j) in enumerate(planes):
            tot = edge(i, ()) + edge(j, (i,)) - edge(i, (j,)) - edge(j, ())
            W[s, k] = np.rint(tot / (2 * pi_l)).astype(np.int64)
    return W


def bruteforce_overlap(anchor, other, tol):
    nz, ny, nx = anchor.shape
    count = 0
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                if anchor[z, y, x] == 0:
                    continue
                hit = False
                for dz in range(-tol, tol + 1):
                    for dy in range(-tol, tol + 1):
                        for dxx in range(-tol, tol + 1):
                            if other[(z + dz) % nz, (y + dy) % ny, (x + dxx) % nx] > 0:
                                hit = True
                count += hit
    return count


# ---- pins -----------------------------------------------------------------

def pin_gauss_conserved():
    """Gauss law (Eqs. 9-10, Sec. IV).  With k_n = 2 e^2 c_n (1 + delta_n) /
    (1 + omega_n), the half-step residual G_n = div E^{n+1/2} - k_n Im[phi^n*
    pi^{n+1/2}] obeys G_n = (1 - omega_n)/(1 + omega_n) G_{n-1} exactly under
    Eqs. 17-26 whenever k_{n-1} (1 - omega_n) = 2 e^2 c_n (1 - delta_n): in a
    flat background, for beta = 0 in any era and for beta = 1 in radiation.
    So a zero residual stays zero and any other is damped by the product of
    (1 - omega)/(1 + omega) (constant for beta = 1)."""
    cases = [dict(m=0.0, beta=1.0), dict(m=0.5, beta=0.0), dict(m=2.0 / 3.0, beta=0.0),
             dict(m=0.5, beta=1.0, eta_ref=7.0)]
    nsteps = 12
    for kw in cases:
        p = O.Params(10, 8, 6, e=(1.0, 0.7), **kw)
        st = synth.random_state(p.shape, seed=11, a_amp=1.0, mom_amp=0.5)
        G = []
        for n in (0, nsteps):
            if n:
                O.step(p, st, 0, n)
            a, c, d, w = step_coefficients(p, n - 1)
            ct = c * (1 + d) / (1 + w)
            G.append([divergence_E(st, s, p.dx) - 2 * p.e[s] ** 2 * ct
                      * np.imag(np.conj(cplx(st, s)) * mom(st, s)) for s in range(2)])
        damp = 1.0
        for n in range(nsteps):
            w = step_coefficients(p, n)[3]
            damp *= (1 - w) / (1 + w)
        d = O.diagnostic_sums(p, st, nsteps)
        for s in range(2):
            scale = np.abs(G[0][s]).max()
            err = np.abs(G[1][s] - damp * G[0][s]).max()
            assert scale > 1e-2, "test state should violate Gauss initially"
            assert err < 1e-11 * max(1.0, scale), (kw, s, err)
            # the oracle's own Gauss diagnostic reports the same residual
            tag = "pq"[s]
            assert abs(d["gauss_max_" + tag] - np.abs(G[1][s]).max()) < 1e-11 * scale
            assert abs(d["gauss_sum_" + tag] - np.abs(G[1][s]).sum()) < 1e-9 * np.abs(G[1][s]).sum()


def pin_gauss_step_identity():
    """Per-step form of the Gauss law valid for every beta and era: with
    D = div E and Q = Im[phi^n* pi],
    (1+omega) D^{n+1/2} - (1-omega) D^{n-1/2}
      = 2 e^2 c_n [(1+delta) Q^{n+1/2} - (1-delta) Q^{n-1/2}]."""
    for kw in (dict(m=2.0 / 3.0, beta=1.0), dict(m=0.5, beta=-1.0), dict(m=2.0 / 3.0, beta=0.4)):
        p = O.Params(8, 10, 6, e=(1.0, 1.3), **kw)
        st = synth.random_state(p.shape, seed=3)
        n = 5
        a, c, d, w = step_coefficients(p, n)
        pi_new, e_new = O.kicks(p, st, n)
        for s in range(2):
            Dm = divergence_E(st, s, p.dx)
            tmp = np.zeros_like(st)
            tmp[14:20] = e_new
            Dp = divergence_E(tmp, s, p.dx)
            f = cplx(st, s)
            Qm = np.imag(np.conj(f) * mom(st, s))
            Qp = np.imag(np.conj(f) * (pi_new[2 * s] + 1j * pi_new[2 * s + 1]))
            R = (1 + w) * Dp - (1 - w) * Dm - 2 * p.e[s] ** 2 * c * ((1 + d) * Qp - (1 - d) * Qm)
            assert np.abs(R).max() < 1e-11 * max(1.0, np.abs(Dp).max()), (kw, s, np.abs(R).max())


def pin_energy_second_order():
    """At a = 1 (flat) the leapfrog conserves the energy
    sum [|pi|^2 + |D^+ phi|^2 + (E^2 + F^2)/(2 e^2) + V] up to bounded
    O(deta^2) oscillations: halving deta divides the maximum deviation by
    about four, with no secular drift."""
    devs = []
    for deta, nsteps in ((0.1, 200), (0.05, 400)):
        p = O.Params(12, 12, 12, m=0.0, deta=deta, kappa=0.5)
        st = synth.smooth_state(p.shape, seed=5, kmax=1, amp=0.2, a_amp=0.2)
        e0 = O.diagnostics(p, st, 0)["energy_total"]
        dev = 0.0
        every = nsteps // 20
        for n in range(0, nsteps, every):
            O.step(p, st, n, every)
            e = O.diagnostics(p, st, n + every)["energy_total"]
            dev = max(dev, abs(e - e0) / e0)
        devs.append(dev)
    ratio = devs[0] / devs[1]
    assert devs[0] < 5e-2, devs
    assert 3.0 < ratio < 5.5, (devs, ratio)


def _discrete_freq(deta, khat2, mass2):
    return 2.0 * math.asin(0.5 * deta * math.sqrt(khat2 + mass2))


def pin_linear_dispersion():
    """Small plane waves about the vacuum phi = psi = sigma at a = 1 follow
    the exact leapfrog dispersion sin^2(W/2) = deta^2 (khat^2 + M^2) / 4 with
    khat^2 = (4/dx^2) sin^2(k dx / 2) and
      M^2 = sigma^2 (lambda -+ 2 kappa)  (in-phase / out-of-phase radial modes,
            from the potential of Eq. 4),
      M^2 = 2 e^2 sigma^2               (transverse gauge mode, Eq. 20)."""
    nx, eps, nsteps = 16, 1e-7, 120
    p = O.Params(nx, 4, 4, m=0.0, kappa=0.9)
    X = np.arange(nx)[None, None, :] * np.ones(p.shape)
    jk = 3
    kdx = TWO_PI * jk / nx
    khat2 = 4.0 / p.dx ** 2 * math.sin(kdx / 2) ** 2
    prof = np.cos(kdx * X)
    sig = p.sigma[0]
    for sgn in (+1, -1):
        mass2 = sig ** 2 * (p.lam[0] - sgn * 2 * p.kappa)
        Wf = _discrete_freq(p.deta, khat2, mass2)
        st = O.new_state(p)
        st[0] = sig + eps * prof
        st[2] = sig + sgn * eps * prof
        st[10] = eps * prof * (1 - math.cos(Wf)) / p.deta
        st[12] = sgn * st[10]
        O.step(p, st, 0, nsteps)
        exp_h = eps * prof * math.cos(nsteps * Wf)
        err = max(np.abs(st[0] - sig - exp_h).max(), np.abs(st[2] - sig - sgn * exp_h).max())
        assert err < 1e-4 * eps, ("scalar", sgn, err / eps)
    mass2 = 2 * p.e[0] ** 2 * sig ** 2
    Wf = _discrete_freq(p.deta, khat2, mass2)
    st = O.new_state(p)
    st[0] = sig
    st[2] = sig
    st[5] = eps * prof           # A_1 varying along x: transverse
    st[15] = eps * prof * (1 - math.cos(Wf)) / p.deta
    O.step(p, st, 0, nsteps)
    err = np.abs(st[5] - eps * prof * math.cos(nsteps * Wf)).max()
    assert err < 1e-4 * eps, ("gauge", err / eps)


def _ode_solution(fun, y0, t0, t1):
    from scipy.integrate import solve_ivp
    sol = solve_ivp(fun, (t0, t1), y0, rtol=1e-11, atol=1e-14, method="DOP853")
    return sol.y[:, -1]


def pin_homogeneous_modes():
    """Homogeneous small oscillations in an expanding background follow the
    continuum equations of Sec. III to O(deta^2):
      h'' + 2 (a'/a) h' = -a^{2 beta} lambda sigma^2 h               (Eq. 13)
      A'' + 2 (1 - beta)(a'/a) A' = -2 e^2 a^{2 beta} sigma^2 A       (Eq. 15)
    compared with an adaptive ODE solution (scipy) that uses a(eta) from the
    cosmic-time integral.  Pins delta (Eq. 19), omega (Eq. 22), the a^{2 beta}
    coupling scaling (Eq. 12) and the mass terms."""
    for m, beta in ((0.5, 1.0), (2.0 / 3.0, 0.0), (0.5, -1.0), (2.0 / 3.0, 0.5)):
        p = O.Params(4, 4, 4, m=m, beta=beta, eta0=1.0, eta_ref=1.5, deta=0.004, kappa=0.0)
        nsteps = 500
        eps = 1e-7
        eta0, eta1 = p.eta0, p.eta0 + nsteps * p.deta

        ex = Expansion(m, p.eta_ref, eta0, eta1)
        H, A = ex.hubble, ex.a

        lam, sig, e2 = p.lam[0], p.sigma[0], p.e[0] ** 2
        # discrete initial data: h^0 = eps, pi^{-1/2} = 0; start the ODE at
        # eta0 with h = eps and h' = half a kick (second-order accurate)
        st = O.new_state(p)
        st[0] = sig + eps
        st[2] = p.sigma[1]
        st[5] = eps                      # homogeneous A_1
        O.step(p, st, 0, nsteps)
        c0 = A(eta0) ** (2 * beta)
        hp0 = -0.5 * p.deta * c0 * lam * sig ** 2 * eps
        ap0 = -0.5 * p.deta * c0 * 2 * e2 * sig ** 2 * eps
        # the leapfrog's pi^{1/2} already contains the first kick; its
        # integer-time derivative is half of that
        y = _ode_solution(lambda t, y: [y[1], -2 * H(t) * y[1] - A(t) ** (2 * beta) * lam * sig ** 2 * y[0]],
                          [eps, hp0], eta0, eta1)
        assert abs((st[0] - sig).mean() - y[0]) < 2e-3 * eps, (m, beta, "scalar", (st[0] - sig).mean() / eps, y[0] / eps)
        y = _ode_solution(lambda t, y: [y[1], -2 * (1 - beta) * H(t) * y[1]
                                        - 2 * e2 * A(t) ** (2 * beta) * sig ** 2 * y[0]],
                          [eps, ap0], eta0, eta1)
        assert abs(st[5].mean() - y[0]) < 2e-3 * eps, (m, beta, "gauge", st[5].mean() / eps, y[0] / eps)


def pin_gauge_covariance():
    """Lattice gauge invariance of the discretisation (Sec. II covariant
    derivatives): stepping a gauge-transformed state equals transforming the
    stepped state; windings, cells and all diagnostic sums are unchanged."""
    p = O.Params(10, 8, 6, m=0.5, beta=1.0, eta_ref=5.0, e=(1.0, 0.6))
    st = synth.random_state(p.shape, seed=21)
    lam = synth.gauge_parameter(p.shape, seed=22)
    g_then_step = O.step(p, gauge_transform(p, st, lam), 0, 3)
    step_then_g = gauge_transform(p, O.step(p, st.copy(), 0, 3), lam)
    err = np.abs(g_then_step - step_then_g).max()
    assert err < 1e-10, err
    W1, F1 = O.windings(p, st)
    W2, F2 = O.windings(p, gauge_transform(p, st, lam))
    ok = (F1 == 0) & (F2 == 0)
    assert np.array_equal(W1[ok], W2[ok])
    d1 = O.diagnostic_sums(p, st, 0)
    d2 = O.diagnostic_sums(p, gauge_transform(p, st, lam), 0)
    for k in d1:
        assert abs(d1[k] - d2[k]) <= 1e-9 * max(1.0, abs(d1[k])), (k, d1[k], d2[k])


def pin_sector_swap():
    """The phi <-> psi, A <-> B exchange symmetry of Sec. II: swapping the
    sectors and their couplings commutes with the step, bit for bit."""
    p = O.Params(8, 6, 10, m=2.0 / 3.0, beta=0.0, lam=(2.0, 1.4), e=(1.0, 0.8), sigma=(1.0, 0.9),
                 kappa=0.5)
    q = O.Params(8, 6, 10, m=2.0 / 3.0, beta=0.0, lam=(1.4, 2.0), e=(0.8, 1.0), sigma=(0.9, 1.0),
                 kappa=0.5)
    st = synth.random_state(p.shape, seed=7)
    a = O.step(p, st.copy(), 0, 4)
    b = swap_sectors(O.step(q, swap_sectors(st), 0, 4))
    assert np.array_equal(a, b)
    da, db = O.diagnostic_sums(p, st, 0), O.diagnostic_sums(q, swap_sectors(st), 0)
    for k in ("energy", "lag", "rl_num", "rl_den"):
        assert abs(da[k] - db[k]) <= 1e-12 * abs(da[k]), k


def pin_kappa_decoupling():
    """With kappa = 0 the potential of Eq. 4 separates and the two sectors are
    independent Abelian-Higgs copies: perturbing p leaves q untouched."""
    p = O.Params(8, 8, 8, m=0.5, beta=1.0, eta_ref=3.0, kappa=0.0)
    st = synth.random_state(p.shape, seed=8)
    st2 = st.copy()
    st2[[0, 1, 4, 5, 6, 10, 11, 14, 15, 16]] += 0.1 * synth.random_state(p.shape, seed=9)[
        [0, 1, 4, 5, 6, 10, 11, 14, 15, 16]]
    a = O.step(p, st, 0, 3)
    b = O.step(p, st2, 0, 3)
    q_fields = [2, 3, 7, 8, 9, 12, 13, 17, 18, 19]
    assert np.array_equal(a[q_fields], b[q_fields])
    assert not np.array_equal(a[[0, 1]], b[[0, 1]])


def pin_winding_topology():
    """Integer topology of plaquette windings (Sec. III.A): on any state the
    oriented winding flux out of every cell is zero (no monopoles), the flux
    through every periodic lattice slice is zero, every cell value is even,
    and the cell values sum to twice the number of pierced plaquettes."""
    p = O.Params(12, 10, 8, m=0.5, beta=1.0, eta_ref=4.0)
    st = O.init(p)
    O.step(p, st, 0, 15)
    W, F = O.windings(p, st)
    C = O.cells(p, W)
    assert np.abs(W).sum() > 20, "state should contain strings"
    for s in range(2):
        w01, w02, w12 = (W[s, k].astype(np.int64) for k in range(3))
        flux = (roll(w01, 1, 2) - w01) - (roll(w02, 1, 1) - w02) + (roll(w12, 1, 0) - w12)
        assert not flux.any()
        assert not w01.sum(axis=(1, 2)).any()     # z-normal flux through each z-plane
        assert not w02.sum(axis=(0, 2)).any()     # y-normal flux through each y-plane
        assert not w12.sum(axis=(0, 1)).any()     # x-normal flux through each x-plane
        assert not (C[s] % 2).any()
        assert int(C[s].astype(np.int64).sum()) == 2 * int(np.abs(W[s]).sum())


def pin_cooling_ignores_background_and_momenta():
    """The cooling flow (Eqs. 27-30) is a flow in flow time at a = 1 with no
    damping and no momenta: cooling a rough state gives bit-identical
    positions whatever the run's era, beta, initial time and time step, and
    whatever its momenta hold."""
    base = dict(lam=(2.0, 1.6), e=(1.0, 0.8), sigma=(1.0, 0.9), kappa=0.4)
    pf = O.Params(6, 6, 6, m=0.0, **base)
    pe = O.Params(6, 6, 6, m=2.0 / 3.0, beta=0.5, eta0=3.0, eta_ref=1.5, deta=0.05, **base)
    st = synth.random_state(pf.shape, seed=7)
    still = st.copy()
    still[10:] = 0.0
    outs = [O.cool(pf, still.copy(), 0.02, 12), O.cool(pe, still.copy(), 0.02, 12), O.cool(pf, st.copy(), 0.02, 12)]
    assert not np.array_equal(outs[0][:10], still[:10])
    for o in outs[1:]:
        assert np.array_equal(o[:10], outs[0][:10])


def pin_double_winding_plaquette():
    """A plaquette of winding -2 (Sec. III.A definition; the census of
    |W| >= 2 plaquettes and of cells of value >= 4).  phi = 1 in both
    sectors and zero links, except the x-link at x0 and the y-link at
    x0 + x of sector p, each of angle dx A = -2 pi + 0.1.  Each of these edges
    has chi = -0.1 and branch integer k = rint((0 - dx A) / 2 pi) = 1, so the
    (x, y) plaquette at x0, which holds both, has W = -(1 + 1) = -2, and each
    of the three other plaquettes on either link has |W| = 1: one plaquette
    of |W| = 2, six of |W| = 1, no flag.  The two cells on either side of the
    W = -2 face also hold one |W| = 1 face of each link: value 4."""
    p = O.Params(6, 6, 6, m=0.0)
    st = O.new_state(p)
    st[0] = 1.0
    st[2] = 1.0
    x0 = (2, 2, 2)  # (z, y, x)
    xx = (2, 2, 3)
    theta = -TWO_PI + 0.1
    st[4][x0] = theta / p.dx
    st[5][xx] = theta / p.dx
    W, F = O.windings(p, st)
    assert not F.any() and not W[1].any()
    assert W[0, 0][x0] == -2
    aw = np.abs(W[0].astype(np.int64))
    assert int((aw == 2).sum()) == 1 and int((aw == 1).sum()) == 6 and int(aw.max()) == 2
    res = O.strings(p, st, tol=1)
    assert res["n_w2_p"] == 1 and res["n_w2_q"] == 0 and res["max_abs_w"] == 2
    assert res["n_cells_ge4_p"] == 2 and res["n_cells_ge4_q"] == 0 and res["n_flagged"] == 0


def pin_branch_cut_flags():
    """Branch-cut flags of the windings (Sec. III.A, with the reading that an
    edge is flagged when its phase chi is within 1e-4 of pi, or when a field
    at either end is exactly zero).  Zero links, phi_q = 1 and phi_p = 1
    except at three sites: one of phase pi - 5e-5, one of phase pi - 1e-3 and
    one of zero field.  Every edge touching the first or the third site has
    pi - |chi| = 5e-5 or a zero product, so exactly the twelve plaquettes with
    either site as a corner are flagged; the second site's edges sit 1e-3
    from the cut and flag nothing.  The phase field is single-valued, so
    every winding is zero."""
    p = O.Params(6, 6, 6, m=0.0)
    st = np.zeros((O.NFIELDS, 6, 6, 6))
    st[0] = 1.0
    st[2] = 1.0
    near, far, zero = (1, 1, 1), (1, 1, 4), (4, 4, 1)  # (z, y, x)
    for site, ph in ((near, math.pi - 5e-5), (far, math.pi - 1e-3)):
        st[0][site], st[1][site] = math.cos(ph), math.sin(ph)
    st[0][zero] = 0.0
    W, F = O.windings(p, st)
    assert not W.any()
    expect = np.zeros(F.shape[1:], dtype=bool)
    for k, (i, j) in enumerate(((0, 1), (0, 2), (1, 2))):  # plane k spans directions i < j (0 = x)
        for corner in (near, zero):
            for a in (0, 1):
                for b in (0, 1):
                    zyx = list(corner)
                    zyx[2 - i] = (zyx[2 - i] - a) % 6
                    zyx[2 - j] = (zyx[2 - j] - b) % 6
                    expect[k][tuple(zyx)] = True
    assert int(expect.sum()) == 24
    assert np.array_equal(F[0].astype(bool), expect)
    assert not F[1].any()


def pin_planted_vortices():
    """Four planted straight strings (synth.vortex_map) are found at exactly
    the plaquettes and with the signs the map fixes, once per z-plane, with
    cell value 2 (Sec. III.B: a unit string pierces two faces), also after a
    random gauge transformation; the cell overlap counts follow from the
    placement of the q strings (same cells, one cell away, two away)."""
    shape = (6, 12, 16)
    nz, ny, nx = shape
    p = O.Params(nx, ny, nz, m=0.0)
    vm = synth.vortex_map(shape)
    expect = np.zeros(shape, dtype=np.int64)
    for (x0, y0, sgn) in ((nx - 1, ny - 1, +1), (nx // 2 - 1, ny - 1, -1),
                          (nx - 1, ny // 2 - 1, -1), (nx // 2 - 1, ny // 2 - 1, +1)):
        expect[:, y0, x0] = sgn
    for shift, want0, want1 in ((0, 4 * nz, 4 * nz), (1, 0, 4 * nz), (2, 0, 0)):
        st = O.new_state(p)
        st[0], st[1] = vm.real, vm.imag
        vq = np.roll(vm, shift, axis=2)
        st[2], st[3] = vq.real, vq.imag
        for variant in ("plain", "gauge"):
            s2 = st if variant == "plain" else gauge_transform(p, st, synth.gauge_parameter(shape, 4))
            W, F = O.windings(p, s2)
            assert not F.any()
            assert np.array_equal(W[0, 0], expect)
            assert np.array_equal(W[1, 0], np.roll(expect, shift, axis=2))
            assert not W[:, 1:].any()
            C = O.cells(p, W)
            assert np.array_equal(C[0], 2 * np.abs(expect))
            assert O.overlap(p, C[0], C[1], 0) == want0
            assert O.overlap(p, C[0], C[1], 1) == want1
        res = O.strings(p, st, tol=1)
        assert res["n_p"] == 4 * nz and res["n_q"] == 4 * nz
        assert res["L_pq"] == p.dx * want1
        assert res["L_p"] == p.dx * (4 * nz) - p.dx * want1
        # the estimators of Eqs. 31-35 from the planted geometry: four strings
        # of length nz dx per sector, bound (within one cell) or not
        vol = nx * ny * nz * p.dx ** 3
        bound = p.dx * want1
        alone = 4 * nz * p.dx - bound  # per sector
        total = 2 * alone + bound

        def sep(length):
            return math.inf if length == 0 else math.sqrt(vol / length)

        for k, v in (("xi_p", sep(alone)), ("xi_q", sep(alone)), ("xi_pq", sep(bound)), ("xi_w", sep(total)),
                     ("f_total", bound / total)):
            assert math.isclose(res[k], v, rel_tol=1e-14) or res[k] == v, (shift, k, res[k], v)
        assert math.isnan(res["f_p"]) if alone == 0 else math.isclose(res["f_p"], bound / alone, rel_tol=1e-14)
    # p strings only (the q sector in its vacuum): the separations of the two
    # sectors differ, so a p/q mix-up in the estimators shows
    st = O.new_state(p)
    st[0], st[1] = vm.real, vm.imag
    st[2] = 1.0
    res = O.strings(p, st, tol=1)
    vol, lp = nx * ny * nz * p.dx ** 3, 4 * nz * p.dx
    assert res["n_q"] == 0 and res["L_pq"] == 0.0 and res["L_p"] == lp
    assert math.isclose(res["xi_p"], math.sqrt(vol / lp), rel_tol=1e-14) and res["xi_q"] == math.inf
    assert res["xi_pq"] == math.inf and math.isclose(res["xi_w"], math.sqrt(vol / lp), rel_tol=1e-14)
    assert res["f_total"] == 0.0 and res["f_p"] == 0.0
    # eight p strings (the map times itself shifted by nx/4, whose zero lines
    # sit four cells from the first map's) and the four q strings of the map:
    # four p strings are bound and four are not, so L_pq = L_p = 4 nz dx,
    # L_q = 0, f_total = 1/2 (Eq. 34) and f_p = 1 (Eq. 35); 4 nz plaquettes
    # are pierced in both sectors
    st = O.new_state(p)
    vp = vm * np.roll(vm, nx // 4, axis=2)
    st[0], st[1] = vp.real, vp.imag
    st[2], st[3] = vm.real, vm.imag
    W, F = O.windings(p, st)
    assert not F.any() and int(np.abs(W[0]).sum()) == 8 * nz and int(np.abs(W[1]).sum()) == 4 * nz
    res = O.strings(p, st, tol=1)
    L4 = 4 * nz * p.dx
    assert res["n_pq_plaq"] == 4 * nz and res["n_pq_cell"] == 4 * nz
    assert res["L_pq"] == L4 and res["L_p"] == L4 and res["L_q"] == 0.0
    assert res["f_total"] == 0.5 and res["f_p"] == 1.0 and res["xi_q"] == math.inf
    assert math.isclose(res["xi_w"], math.sqrt(vol / (2 * L4)), rel_tol=1e-14)
    # the same eight p strings against the four q strings of the map shifted
    # by two cells: within two cells every p string has a q string, and each
    # q string has two p strings, so the p-anchored count is 8 nz cells and
    # the q-anchored one 4 nz (Sec. III.B); within one cell neither has any
    vq = np.roll(vm, 2, axis=2)
    st[2], st[3] = vq.real, vq.imag
    res2 = O.strings(p, st, tol=2)
    assert res2["n_pq_cell"] == 8 * nz and res2["n_pq_cell_q"] == 4 * nz
    res1 = O.strings(p, st, tol=1)
    assert res1["n_pq_cell"] == 0 and res1["n_pq_cell_q"] == 0


def pin_bruteforce_windings():
    """Windings on rough random 8^3 states agree with an independent
    per-site-phase count (bruteforce_windings) on every unflagged plaquette,
    and the overlap count agrees with a 27-neighbour loop."""
    p = O.Params(8, 8, 8, m=0.0)
    for seed in (1, 2, 3):
        st = synth.random_state(p.shape, seed=seed, a_amp=4.0)
        W, F = O.windings(p, st)
        Wb = bruteforce_windings(p, st)
        ok = F == 0
        assert np.array_equal(W[ok].astype(np.int64), Wb[ok])
        assert np.abs(W).max() >= 1
        C = O.cells(p, W)
        for tol in (0, 1):
            assert O.overlap(p, C[0], C[1], tol) == bruteforce_overlap(C[0], C[1], tol)
            assert O.overlap(p, C[1], C[0], tol) == bruteforce_overlap(C[1], C[0], tol)


def pin_velocity_closed_form():
    """Eqs. 36-37 on a travelling phase wave phi_s = r_s e^{i k x},
    pi_s^{n-1/2} = i v khat phi_s, A = E = 0 at a = 1: every site is alike,
    so for either weight R = sum_s r_s^2 (v^2 khat^2 + deta^2 (khat^2 + g_s)^2 / 2)
    / (khat^2 sum_s r_s^2), with g_s = lambda_s/2 (r_s^2 - sigma_s^2)
    - kappa (r_o^2 - sigma_o^2) the radial force of Eq. 17."""
    nx = 16
    p = O.Params(nx, 4, 4, m=0.0, kappa=0.7, lam=(2.0, 1.6))
    r = (0.8, 1.1)
    v = 0.3
    kdx = TWO_PI * 2 / nx
    khat2 = 4.0 / p.dx ** 2 * math.sin(kdx / 2) ** 2
    X = np.arange(nx)[None, None, :] * np.ones(p.shape)
    st = O.new_state(p)
    for s in range(2):
        f = r[s] * np.exp(1j * kdx * X)
        pm = 1j * v * math.sqrt(khat2) * f
        st[2 * s], st[2 * s + 1] = f.real, f.imag
        st[10 + 2 * s], st[11 + 2 * s] = pm.real, pm.imag
    d = O.diagnostics(p, st, 0)
    num = 0.0
    for s in range(2):
        o = 1 - s
        g = 0.5 * p.lam[s] * (r[s] ** 2 - p.sigma[s] ** 2) - p.kappa * (r[o] ** 2 - p.sigma[o] ** 2)
        num += r[s] ** 2 * (v * v * khat2 + 0.5 * p.deta ** 2 * (khat2 + g) ** 2)
    R = num / (khat2 * (r[0] ** 2 + r[1] ** 2))
    assert abs(d["R_l"] - R) < 1e-11 * R, (d["R_l"], R)
    assert abs(d["R_pq"] - R) < 1e-11 * R, (d["R_pq"], R)
    assert abs(d["v2_l"] - 2 * R / (1 + R)) < 1e-11
    assert abs(d["grad_p"] - p.nsites * r[0] ** 2 * khat2) < 1e-10 * p.nsites
    # the potential of Eq. 4 at a = 1, the same at every site
    rp, rq = r[0] ** 2 - p.sigma[0] ** 2, r[1] ** 2 - p.sigma[1] ** 2
    vp, vq = p.lam[0] / 4 * rp * rp, p.lam[1] / 4 * rq * rq
    for k, want in (("pot", vp + vq - p.kappa * rp * rq), ("pot_p", vp), ("pot_q", vq), ("vint", p.kappa * rp * rq)):
        assert abs(d[k] - p.nsites * want) < 1e-12 * p.nsites * max(abs(want), 1e-3), (k, d[k], p.nsites * want)
    for s, sec in enumerate("pq"):
        assert abs(d["phi_min_" + sec] - r[s]) < 1e-14 and abs(d["phi_max_" + sec] - r[s]) < 1e-14
    # kappa = 0: every V_int weight of Eq. 37 vanishes, so <v^2> weighted by
    # V_int is undefined while the L-weighted one keeps its closed form
    p0 = O.Params(nx, 4, 4, m=0.0, kappa=0.0, lam=(2.0, 1.6))
    d0 = O.diagnostics(p0, st, 0)
    num0 = sum(r[s] ** 2 * (v * v * khat2 + 0.5 * p0.deta ** 2
                            * (khat2 + 0.5 * p0.lam[s] * (r[s] ** 2 - p0.sigma[s] ** 2)) ** 2) for s in range(2))
    R0 = num0 / (khat2 * (r[0] ** 2 + r[1] ** 2))
    assert abs(d0["R_l"] - R0) < 1e-11 * R0, (d0["R_l"], R0)
    assert math.isnan(d0["R_pq"]) and math.isnan(d0["v2_pq"])


def pin_homogeneous_energy_expanding():
    """The lattice energy densities with their a^{2 beta} factors (the action
    of Sec. II; V of Eq. 4) on a homogeneous state in an expanding background:
    matter era (a ~ eta^2), beta = 1/2, eta = 2 eta_ref, so a = 4 and
    c = a^{2 beta} = 4.  Uniform real phi_s = r_s off the vacuum, uniform
    imaginary momenta pi_s = i u_s, A = 0 and a uniform electric field per
    sector: no gradient, no current, no curl.  The kicks of Eqs. 17 and 20
    then give pi_s^+ = ((1 - delta) pi_s^- - deta c g_s r_s) / (1 + delta)
    with g_s = lambda_s/2 (r_s^2 - sigma_s^2) - kappa (r_o^2 - sigma_o^2),
    and E^+ = (1 - omega) / (1 + omega) E^-, and every lattice sum is V times
    the site value: kin_s = (|pi^-|^2 + |pi^+|^2) / 2,
    el_s = sum_i (E_i^-2 + E_i^+2) / 2 / (2 e_s^2 c), pot = c V(r_p, r_q),
    grad = mag = 0, L = sum (kin + el) - pot, H = sum (kin + el) + pot."""
    p = O.Params(4, 4, 4, m=2.0 / 3.0, beta=0.5, eta0=2.0, eta_ref=1.0, kappa=0.3, lam=(2.0, 1.6),
                 e=(1.0, 0.8), sigma=(1.0, 0.9))
    cf = O.coeffs(p, 0)
    c = (p.eta0 / p.eta_ref) ** (2.0 * p.beta * p.m / (1.0 - p.m))
    assert abs(cf["a"] - 4.0) < 1e-14 and abs(cf["c"] - c) < 1e-14 * c and abs(c - 4.0) < 1e-14
    delta, omega = cf["delta"], cf["omega"]
    assert delta > 0.0 and omega > 0.0
    r, u = (0.8, 1.2), (0.3, -0.2)
    E = ((0.4, -0.1, 0.25), (-0.3, 0.2, 0.15))
    st = O.new_state(p)
    for s in range(2):
        st[2 * s] = r[s]
        st[11 + 2 * s] = u[s]
        for i in range(3):
            st[14 + 3 * s + i] = E[s][i]
    d = O.diagnostics(p, st, 0)
    V = p.nsites
    rr = [r[s] ** 2 - p.sigma[s] ** 2 for s in range(2)]
    q = (1.0 - omega) / (1.0 + omega)
    kin, el = [], []
    for s in range(2):
        g = 0.5 * p.lam[s] * rr[s] - p.kappa * rr[1 - s]
        pr_plus = -p.deta * c * g * r[s] / (1.0 + delta)
        pi_plus = (1.0 - delta) * u[s] / (1.0 + delta)
        kin.append(0.5 * (u[s] ** 2 + pr_plus ** 2 + pi_plus ** 2))
        el.append(sum(x * x for x in E[s]) * (1.0 + q * q) / 2.0 / (2.0 * p.e[s] ** 2 * c))
    pot = c * (p.lam[0] / 4 * rr[0] ** 2 + p.lam[1] / 4 * rr[1] ** 2 - p.kappa * rr[0] * rr[1])
    want = dict(kin_p=kin[0], kin_q=kin[1], el_p=el[0], el_q=el[1], pot=pot,
                lag=kin[0] + kin[1] + el[0] + el[1] - pot, energy=kin[0] + kin[1] + el[0] + el[1] + pot)
    for k, w in want.items():
        assert abs(d[k] - V * w) < 1e-12 * V * abs(w), (k, d[k], V * w)
    for k in ("grad_p", "grad_q", "mag_p", "mag_q"):
        assert d[k] == 0.0, (k, d[k])


def pin_vacuum():
    """Special values: in the vacuum every force vanishes, there are no
    windings, string lengths are zero so the separations are infinite and the
    fractions undefined."""
    p = O.Params(8, 8, 8, m=0.5, beta=1.0, eta_ref=2.0)
    st = O.new_state(p)
    st[0] = 1.0
    st[2] = 1.0
    pi_new, e_new = O.kicks(p, st, 3)
    assert not pi_new.any() and not e_new.any()
    res = O.strings(p, st)
    assert res["n_p"] == 0 and res["n_q"] == 0 and res["n_pq_cell"] == 0
    assert math.isinf(res["xi_w"]) and math.isnan(res["f_total"])
    d = O.diagnostics(p, st, 3)
    assert d["energy"] == 0.0 and d["lag"] == 0.0


def pin_string_tension():
    """Criticality (Eq. 11, lambda = 2 e^2, sigma = 1): a straight vortex has
    tension 2 pi sigma^2.  The four planted strings of synth.vortex_map,
    relaxed with the cooling flow of Eqs. 27-30 (kappa = 0), have static
    energy per unit length 4 x 2 pi within the O(dx^2) lattice error, which
    shrinks as dx does."""
    errs = []
    for dx, n, iters in ((0.5, 24, 600), (0.35, 34, 1200)):
        p = O.Params(n, n, 2, dx=dx, m=0.0, kappa=0.0, lam=(2.0, 2.0), e=(1.0, 1.0))
        st = O.new_state(p)
        f = synth.vortex_map(p.shape)
        st[0], st[1] = f.real, f.imag
        st[2] = 1.0
        O.cool(p, st, 0.16 * dx * dx, iters)
        W, _ = O.windings(p, st)
        assert int(np.abs(W[0, 0]).sum()) == 4 * p.nz
        d = O.diagnostics(p, st, 0)
        e_static = p.dx ** 3 * (d["grad_p"] + d["mag_p"] + d["pot"])
        tension = e_static / (p.nz * p.dx) / 4.0
        errs.append(abs(tension / TWO_PI - 1.0))
        # a relaxed static network has L = -(energy density) (Eq. 33's premise)
        # and xi_L = sqrt(V / total string length) up to the tension error
        assert abs(d["lag_total"] + e_static) < 1e-6 * e_static, (d["lag_total"], e_static)
        assert abs(d["energy_total"] - e_static) < 1e-6 * e_static
        vol = p.nsites * p.dx ** 3
        assert abs(d["xi_l"] / math.sqrt(vol / (4 * p.nz * p.dx)) - 1.0) < 0.02
    assert errs[0] < 0.03, errs
    assert errs[1] < 0.7 * errs[0], errs


def pin_unequal_tensions():
    """Unequal tensions (the next step the paper names, Sec. VI): with
    sigma_p = 1.1, sigma_q = 0.8 and lambda_s = 2 e_s^2 the strings of both
    sectors are BPS with tension 2 pi sigma_s^2; after cooling, each
    sector's static energy per length is 4 x 2 pi sigma_s^2 within the
    lattice and finite-box error, and its Lagrangian separation
    xi_L,s = sqrt(-mu_s V / L_s), mu_s = 2 pi sigma_s^2, equals the winding
    separation sqrt(V / L) of its four planted strings.  The whole network's
    xi_L (mu = 2 pi sigma_p^2 over both sectors' Lagrangian, which for
    static strings is minus their energy) is then
    sqrt(V / L * sigma_p^2 / (sigma_p^2 + sigma_q^2))."""
    n, dx = 32, 0.5
    p = O.Params(n, n, 2, dx=dx, m=0.0, kappa=0.0, lam=(2.0, 1.62), e=(1.0, 0.9), sigma=(1.1, 0.8))
    st = O.new_state(p)
    f = synth.vortex_map(p.shape, sigma=1.1)
    g = synth.vortex_map(p.shape, sigma=0.8)
    st[0], st[1], st[2], st[3] = f.real, f.imag, g.real, g.imag
    O.cool(p, st, 0.15 * dx * dx, 960)  # forward Euler stays stable for the stiffest mode
    d = O.diagnostics(p, st, 0)
    vol = p.nsites * dx ** 3
    length = 4 * p.nz * dx
    for k, sec in enumerate("pq"):
        e_static = dx ** 3 * (d["grad_" + sec] + d["mag_" + sec] + d["pot_" + sec])
        tension = e_static / length
        assert abs(tension / (TWO_PI * p.sigma[k] ** 2) - 1.0) < 0.02, (sec, tension)
        assert abs(d["xi_l_" + sec] / math.sqrt(vol / length) - 1.0) < 0.01, sec
    sp2, sq2 = p.sigma[0] ** 2, p.sigma[1] ** 2
    assert abs(d["xi_l"] / math.sqrt(vol / length * sp2 / (sp2 + sq2)) - 1.0) < 0.01


def pin_higher_winding_census():
    """Cells carrying more than one unit of winding (value >= 4, the
    signature of a (2,0) string, Sec. III.B): four z-strings crossing four
    x-strings (synth.crossing_vortices) share exactly 8 cells, which read 4;
    every other pierced cell reads 2 and no plaquette carries |W| >= 2."""
    shape = (8, 12, 16)
    nz, ny, nx = shape
    p = O.Params(nx, ny, nz, m=0.0)
    st = O.new_state(p)
    f = synth.crossing_vortices(shape)
    st[0], st[1] = f.real, f.imag
    st[2] = 1.0
    r = O.strings(p, st)
    assert r["n_p"] == 4 * nz + 4 * nx and r["max_abs_w"] == 1
    assert r["n_w2_p"] == 0 and r["n_cells_ge4_p"] == 8 and r["n_cells_ge4_q"] == 0
    vals, counts = np.unique(r["cells"][0], return_counts=True)
    assert set(vals.tolist()) == {0, 2, 4} and counts[list(vals).index(4)] == 8


def pin_random_phase_ic():
    """Initial conditions of Sec. III: |phi_s| = sigma_s at every site with a
    uniform random phase (Kolmogorov-Smirnov test against U[0, 2 pi)),
    independent between sectors and seeds, all other fields zero."""
    from scipy.stats import kstest
    p = O.Params(16, 16, 16, sigma=(1.0, 0.8), seed=12345)
    st = O.init(p)
    assert not st[4:].any()
    th = []
    for s in range(2):
        f = cplx(st, s)
        assert np.abs(np.abs(f) - p.sigma[s]).max() < 1e-15
        t = np.mod(np.angle(f), TWO_PI).ravel()
        assert kstest(t / TWO_PI, "uniform").pvalue > 1e-4
        th.append(t)
    assert abs(np.corrcoef(np.cos(th[0]), np.cos(th[1]))[0, 1]) < 0.05
    q = O.Params(16, 16, 16, sigma=(1.0, 0.8), seed=12346)
    other = np.mod(np.angle(cplx(O.init(q), 0)), TWO_PI).ravel()
    assert abs(np.corrcoef(np.cos(th[0]), np.cos(other))[0, 1]) < 0.05
    assert np.array_equal(O.init(p), st)


def pin_bruteforce_overlap():
    """The fast cell-overlap count of Sec. III.B on sparse random cell arrays
    (5% occupancy, so that the displacement direction matters) agrees with a
    direct loop over the (2 tol + 1)^3 neighbourhood for tol = 0, 1, 2, in
    both anchorings."""
    p = O.Params(10, 9, 8)
    for seed in (1, 2):
        a = synth.sparse_cells(p.shape, 0.05, seed)
        b = synth.sparse_cells(p.shape, 0.05, seed + 100)
        for tol in (0, 1, 2):
            assert O.overlap(p, a, b, tol) == bruteforce_overlap(a, b, tol)
            assert O.overlap(p, b, a, tol) == bruteforce_overlap(b, a, tol)


def bruteforce_components(mask):
    """Periodic 26-connected labelling by repeated relaxation: every cell takes
    the smallest label among itself and its 26 neighbours until nothing
    changes (labels start as the site indices)."""
    nz, ny, nx = mask.shape
    big = np.iinfo(np.int64).max
    lab = np.where(mask > 0, np.arange(mask.size).reshape(mask.shape), big)
    while True:
        best = lab.copy()
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    sh = np.roll(lab, (dz, dy, dx), axis=(0, 1, 2))
                    best = np.minimum(best, np.where(mask > 0, sh, big))
        best = np.where(mask > 0, best, big)
        if np.array_equal(best, lab):
            return np.where(mask > 0, lab, -1)
        lab = best


def pin_components():
    """Connected components of cell masks (the robust method's connectivity
    filter, Sec. III.B): agree with an independent relaxation labelling on
    random periodic masks; cells touching only at a corner are joined
    (26-connectivity); the pq mask agrees with the overlap count."""
    p = O.Params(9, 8, 7)
    for seed, dens in ((1, 0.08), (2, 0.2), (3, 0.35)):
        rng = np.random.default_rng(seed)
        m = (rng.random(p.shape) < dens).astype(np.uint8)
        assert np.array_equal(O.components(p, m), bruteforce_components(m))
    m = np.zeros(p.shape, dtype=np.uint8)
    m[1, 1, 1] = m[2, 2, 2] = 1          # corner contact
    m[5, 6, 8] = m[5, 6, 0] = 1          # face contact across the periodic x boundary
    lab = O.components(p, m)
    assert lab[2, 2, 2] == lab[1, 1, 1] and lab[5, 6, 0] == lab[5, 6, 8]
    assert len(np.unique(lab[lab >= 0])) == 2
    a = synth.sparse_cells(p.shape, 0.1, 5)
    b = synth.sparse_cells(p.shape, 0.1, 6)
    for tol in (0, 1):
        assert int(O.pq_mask(p, a, b, tol).sum()) == O.overlap(p, a, b, tol)


def pin_segments_planted():
    """Four planted straight strings in both sectors (synth.vortex_map): the
    pq cells form four periodic lines of nz cells, so there are four segments
    of length (nz - 1) dx each (Eq. 38 with the off-by-one correction) when
    nz exceeds the threshold, none otherwise."""
    shape = (14, 12, 16)
    nz, ny, nx = shape
    p = O.Params(nx, ny, nz, m=0.0)
    st = O.new_state(p)
    vm = synth.vortex_map(shape)
    st[0], st[1], st[2], st[3] = vm.real, vm.imag, vm.real, vm.imag
    r = O.segments(p, st, tol=1, min_cells=10)
    assert r["n_cells"] == 4 * nz and r["n_components"] == 4 and r["n_segments"] == 4
    assert r["L_pq"] == 4 * (nz - 1) * p.dx and r["l_pq"] == (nz - 1) * p.dx
    assert O.segments(p, st, tol=1, min_cells=nz)["n_segments"] == 0


def pin_cooling_homogeneous_flow():
    """Cooling flow (Eqs. 27-30, read with sigma^2 and without a kappa term):
    for a spatially constant scalar of each sector and zero links, the
    covariant Laplacian and the current vanish, so a forward-Euler step of
    size dt is exactly phi -> phi (1 - dt (lambda_s / 2)(|phi|^2 - sigma_s^2))
    in each sector on its own, whatever kappa and the other sector are.
    Unequal couplings and kappa != 0 make a sector mix-up, a kappa term, a
    wrong factor or sign, or sigma in place of sigma^2 change the result; the
    links stay zero.  600 steps are checked against the same recurrence."""
    p = O.Params(4, 4, 4, m=0.0, lam=(2.0, 1.3), e=(1.0, 0.7), sigma=(1.0, 0.6), kappa=0.45)
    st = np.zeros((20,) + p.shape)
    phi0 = (0.5 * np.exp(0.3j), 1.5 * np.exp(-1.1j))  # |phi| far from each sigma
    for s, f in enumerate(phi0):
        st[2 * s] = f.real
        st[2 * s + 1] = f.imag
    dt, steps = 0.05, 600
    want = list(phi0)
    for k in range(steps):
        for s in range(2):
            r = abs(want[s]) ** 2 - p.sigma[s] ** 2
            want[s] = want[s] * (1.0 - dt * 0.5 * p.lam[s] * r)
        if k == 0:
            one = O.cool(p, st.copy(), dt, 1)
            for s in range(2):
                got = one[2 * s] + 1j * one[2 * s + 1]
                assert np.abs(got - want[s]).max() <= 1e-15 * abs(want[s]), (s, got.flat[0], want[s])
    out = O.cool(p, st, dt, steps)
    for s in range(2):
        got = out[2 * s] + 1j * out[2 * s + 1]
        assert np.abs(got - want[s]).max() <= 1e-12 * abs(want[s]), (s, got.flat[0], want[s])
    assert not out[4:10].any()
    # the flow ends at the vacuum of each sector: |phi_s| -> sigma_s
    assert abs(abs(want[0]) - p.sigma[0]) < 1e-3 and abs(abs(want[1]) - p.sigma[1]) < 1e-3


ALL_PINS = [
    pin_gauss_conserved, pin_gauss_step_identity, pin_energy_second_order,
    pin_linear_dispersion, pin_homogeneous_modes, pin_gauge_covariance, pin_sector_swap,
    pin_kappa_decoupling, pin_winding_topology, pin_planted_vortices, pin_bruteforce_windings, pin_bruteforce_overlap,
    pin_velocity_closed_form, pin_vacuum, pin_string_tension, pin_random_phase_ic, pin_components,
    pin_segments_planted, pin_unequal_tensions, pin_higher_winding_census, pin_cooling_homogeneous_flow,
    pin_branch_cut_flags, pin_homogeneous_energy_expanding, pin_cooling_ignores_background_and_momenta,
    pin_double_winding_plaquette,
]
