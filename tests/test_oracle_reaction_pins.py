"""Pins of the oracle's reaction terms by their dynamics, not by their formulas.

An equilibrium does not see a rate factor (gamma, eps, rho multiply the whole
reaction), so equilibrium checks alone cannot catch a dropped or doubled
factor.  These tests linearise each model by hand about an equilibrium and
compare the oracle's ETD2RKds solution of a small perturbation with the
linear prediction.

* Spatially uniform perturbation (the k = 0 mode).  Every A_mu has zero row
  sums, so K U = 0 and phi_ell(tau A_mu) 1 = 1 / ell!.  One step of Eq. 11
  then reduces to Heun's method for the reaction ODE:
      U2 = U + tau G(U),  U+ = U + tau/2 (G(U) + G(U2))
  (the 2^(d-1) of stage 2 cancels against (1/2)^d of phi_2).  A perturbation
  delta therefore evolves as R(tau J)^n delta with R(Z) = I + Z + Z^2/2, and
  over a horizon T as e^(T J) delta up to the scheme's O(tau^2) error.
* Single cosine mode (Sec. 4.1: the Schnakenberg equilibrium is Turing
  unstable).  cos(k pi i/(n-1)) is an eigenvector of the vertex-grid
  Neumann matrix with eigenvalue 2 delta/h^2 (cos(k pi/(n-1)) - 1), so the
  mode amplitude evolves by e^(T (J + diag(delta^u, delta^v) mu_k)).

J is differentiated by hand from the model equations (Sec. 4.1 Eq. 12,
Sec. 4.2 Eq. 13, Sec. 4.4 Eq. 15, Sec. 4.6 Eq. 17) and written below as
numbers.  A planted mistake (dropped gamma / eps / rho, u^2 v -> u v) fails
these checks: see test_planted_reaction_mistakes_fail.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sl

import workloads as wl
from oracle import schemes

# Schnakenberg with a + b != 1 (so u_e != 1 and u^2 v differs from u v at
# the equilibrium): gamma = 3, a = 0.2, b = 1.3; u_e = a + b = 1.5,
# v_e = b/(a+b)^2.  dg^u/du = gamma(-1 + 2 u v) = 3 * 11/15, dg^u/dv =
# gamma u^2 = 3 * 2.25, dg^v/du = -2 gamma u v = -3 * 26/15, dg^v/dv = -3*2.25.
SCHNAK = dict(model=wl.SCHNAKENBERG, params=(3.0, 0.2, 1.3), ue=1.5, ve=1.3 / 2.25,
              J=[[2.2, 6.75], [-5.2, -6.75]], tau=1e-3, nsteps=1000)
# FitzHugh-Nagumo with eps = 0.05, a1 = 2, a0 = -0.03: the equilibrium solves
# v = u - u^3 and u - a1 v - a0 = 0, i.e. 2 u^3 - u + 0.03 = 0 (small root);
# J = [[1 - 3u^2, -1], [eps, -eps a1]].
_r = np.roots([2.0, 0.0, -1.0, 0.03])
_uf = float(np.real(_r[np.argmin(np.abs(_r))]))
FHN = dict(model=wl.FHN, params=(0.05, 2.0, -0.03), ue=_uf, ve=_uf - _uf ** 3,
           J=[[1.0 - 3.0 * _uf * _uf, -1.0], [0.05, -0.1]], tau=5e-3, nsteps=400)
# FitzHugh-Nagumo of Eq. 13 (rho = 65.731, a1 = 11, a2 = 0.1) about (0, 0):
# J = [[rho, -rho], [rho a1, -rho a1 a2]].
FHN_RHO = dict(model=wl.FHN_RHO, params=(65.731, 11.0, 0.1), ue=0.0, ve=0.0,
               J=[[65.731, -65.731], [723.041, -72.3041]], tau=2.5e-5, nsteps=800)
# DIB of Eq. 15 with the paper's parameters about (0, a4u = 0.5); a4v =
# 1.35/0.55.  dg^u/du = rho a1u (1 - v) = 31.25; dg^u/dv = -rho a3u = -412.5;
# dg^v/du = rho (a1v a2v (1-v)(1 - a3v(1-v)) - a4v a5v v (1 + a3v v))
#         = 6.25 (3.375 - 2.025) = 8.4375;
# dg^v/dv = rho (a1v (-(1 - a3v(1-v)) + a3v (1-v)) - a4v (1 + 2 a3v v))
#         = 6.25 (-2.4 - 1.2 * 1.35/0.55).
DIB = dict(model=wl.DIB, params=tuple(wl.dib_parameters()), ue=0.0, ve=0.5,
           J=[[31.25, -412.5], [8.4375, 6.25 * (-2.4 - 1.2 * 1.35 / 0.55)]], tau=1e-4,
           nsteps=1000)
# Brusselator of Eq. 17 (a = 1, b = 3) about (a, b/a): J = [[b - 1, a^2], [-b, -a^2]].
BRUSS = dict(model=wl.BRUSSELATOR, params=(1.0, 3.0), ue=1.0, ve=3.0,
             J=[[2.0, 1.0], [-3.0, -1.0]], tau=5e-3, nsteps=400)

CASES = {"schnakenberg": SCHNAK, "fhn": FHN, "fhn_rho": FHN_RHO, "dib": DIB,
         "brusselator": BRUSS}


def check_uniform_linearisation(c):
    """Evolve equilibrium + delta0 (spatially constant) with the oracle and
    compare with the hand-derived linearisation, discrete and continuous."""
    p = wl.Problem(d=2, n=(5, 4), lo=(0.0, 0.0), hi=(1.0, 1.0), diff=(1.0, 10.0),
                   adv=((0.3, 0.1), (0.2, -0.4)), model=c["model"], params=c["params"],
                   tau=c["tau"], nsteps=c["nsteps"])
    plan = schemes.make_plan(p)
    d0 = np.array([1e-7, -0.7e-7])
    U = np.full(p.shape, c["ue"] + d0[0])
    V = np.full(p.shape, c["ve"] + d0[1])
    U, V = schemes.etd2rkds_solve(plan, U, V, c["nsteps"])
    # the state stays spatially constant (K const = 0)
    assert np.ptp(U) <= 1e-12 and np.ptp(V) <= 1e-12
    dn = np.array([U.mean() - c["ue"], V.mean() - c["ve"]])
    J = np.array(c["J"])
    tJ = c["tau"] * J
    heun = np.linalg.matrix_power(np.eye(2) + tJ + tJ @ tJ / 2.0, c["nsteps"]) @ d0
    flow = sl.expm(c["nsteps"] * tJ) @ d0
    e_heun = np.linalg.norm(dn - heun) / np.linalg.norm(heun)
    e_flow = np.linalg.norm(dn - flow) / np.linalg.norm(flow)
    # discrete: exact up to the O(|delta|) nonlinear terms and rounding
    assert e_heun <= 1e-5, (e_heun, dn, heun)
    # continuous: the scheme's O(tau^2) global error (tau |lambda| <= 0.01)
    assert e_flow <= 1e-4, (e_flow, dn, flow)


@pytest.mark.parametrize("name", sorted(CASES))
def test_uniform_mode_follows_hand_jacobian(name):
    check_uniform_linearisation(CASES[name])


def test_fhn_growth_rate_is_jacobian_eigenvalue():
    """The FitzHugh-Nagumo variant's near-zero equilibrium is unstable to
    uniform perturbations: the fitted growth rate of log|delta| matches the
    positive eigenvalue of the hand Jacobian (about 0.95)."""
    c = FHN
    p = wl.Problem(d=2, n=(4, 4), lo=(0.0, 0.0), hi=(1.0, 1.0), diff=(1.0, 20.0),
                   adv=((0.5, 0.5), (0.5, 0.5)), model=c["model"], params=c["params"],
                   tau=2e-3, nsteps=1)
    plan = schemes.make_plan(p)
    U = np.full(p.shape, c["ue"] + 1e-9)
    V = np.full(p.shape, c["ve"])
    amps = []
    schemes.etd2rkds_solve(plan, U, V, 4000,
                           callback=lambda n, X, Y: amps.append(
                               (n, math.hypot(X.mean() - c["ue"], Y.mean() - c["ve"]))))
    t = np.array([a[0] for a in amps[2000:]]) * 2e-3
    la = np.log([a[1] for a in amps[2000:]])
    rate = np.polyfit(t, la, 1)[0]
    lam = max(np.linalg.eigvals(np.array(c["J"])).real)
    assert abs(rate - lam) <= 1e-3 * lam, (rate, lam)


def _mode_run(k, n1=40, T=0.05, nsteps=5000):
    """Schnakenberg of Sec. 4.1 (delta^u = 1, delta^v = 10, rho = 1000,
    a^u = 0.1, a^v = 0.9) on [0, 1] x [0, 1], a cosine mode k in x_1."""
    p = wl.Problem(d=2, n=(n1, 3), lo=(0.0, 0.0), hi=(1.0, 1.0), diff=(1.0, 10.0),
                   adv=((0.0, 0.0), (0.0, 0.0)), model=wl.SCHNAKENBERG,
                   params=(1000.0, 0.1, 0.9), tau=T / nsteps, nsteps=nsteps)
    plan = schemes.make_plan(p)
    cosk = np.cos(k * math.pi * np.arange(n1) / (n1 - 1))
    d0 = np.array([1e-7, -0.6e-7])
    ue, ve = 1.0, 0.9
    U = ue + d0[0] * np.broadcast_to(cosk, p.shape)
    V = ve + d0[1] * np.broadcast_to(cosk, p.shape)
    U, V = schemes.etd2rkds_solve(plan, U, V, nsteps)
    w = np.ones(n1)
    w[0] = w[-1] = 0.5
    proj = lambda X: np.sum(w * X[1] * cosk) / np.sum(w * cosk * cosk)  # noqa: E731
    amp = np.array([proj(U - ue), proj(V - ve)])
    h = 1.0 / (n1 - 1)
    mu = 2.0 / h ** 2 * (math.cos(k * math.pi / (n1 - 1)) - 1.0)
    # hand Jacobian at (1, 0.9): 1000 [[-1 + 2uv, u^2], [-2uv, -u^2]]
    M = np.array([[800.0, 1000.0], [-1800.0, -1000.0]]) + np.diag([1.0 * mu, 10.0 * mu])
    return amp, sl.expm(T * M) @ d0, np.linalg.eigvals(M), d0


def test_schnakenberg_turing_mode_grows_at_predicted_rate():
    """Sec. 4.1: the Schnakenberg equilibrium is susceptible of Turing
    instability.  Mode k = 5 (mu_5 ~ -243, inside the unstable band
    200 < -mu < 500 of the hand Jacobian) grows at the rate of
    eig(J + mu D) ~ 38; the uniform mode decays."""
    amp, pred, ev, d0 = _mode_run(5)
    assert max(ev.real) > 30.0
    assert np.linalg.norm(amp) > 4.0 * np.linalg.norm(d0)
    assert np.linalg.norm(amp - pred) <= 1e-3 * np.linalg.norm(pred), (amp, pred)
    amp0, pred0, ev0, _ = _mode_run(0, nsteps=5000)
    assert max(ev0.real) < 0.0
    assert np.linalg.norm(amp0 - pred0) <= 1e-2 * np.linalg.norm(pred0), (amp0, pred0)


def _planted(kind):
    """Reaction functions with one plausible mistake each."""
    def fn(model, params, U, V):
        if kind == "schnak_no_gamma":
            g, a, b = params[:3]
            return a - U + U * U * V, b - U * U * V
        if kind == "schnak_uv":
            g, a, b = params[:3]
            return g * (a - U + U * V), g * (b - U * V)
        if kind == "fhn_no_eps":
            e, a1, a0 = params[:3]
            return U - U ** 3 - V, U - a1 * V - a0
        if kind == "fhn_rho_no_rho":
            r, a1, a2 = params[:3]
            return -U * (U * U - 1.0) - V, r * a1 * (U - a2 * V)
        if kind == "dib_no_rho":
            r, a1u, a2u, a3u, a4u, a1v, a2v, a3v, a4v, a5v = params[:10]
            gu = a1u * (1.0 - V) * U - a2u * U ** 3 - a3u * (V - a4u)
            gv = r * (a1v * (1.0 + a2v * U) * (1.0 - V) * (1.0 - a3v * (1.0 - V))
                      - a4v * V * (1.0 + a5v * U) * (1.0 + a3v * V))
            return gu, gv
        raise ValueError(kind)
    return fn


@pytest.mark.parametrize("kind,case", [("schnak_no_gamma", "schnakenberg"),
                                       ("schnak_uv", "schnakenberg"),
                                       ("fhn_no_eps", "fhn"),
                                       ("fhn_rho_no_rho", "fhn_rho"),
                                       ("dib_no_rho", "dib")])
def test_planted_reaction_mistakes_fail(monkeypatch, kind, case):
    """Each planted mistake in the oracle's reaction makes the uniform-mode
    pin above fail, so that pin really checks the rate factors."""
    monkeypatch.setattr(schemes, "reaction", _planted(kind))
    with pytest.raises(AssertionError):
        check_uniform_linearisation(CASES[case])


def test_planted_gamma_breaks_turing_pin(monkeypatch):
    """The cosine-mode pin also sees a dropped Schnakenberg gamma."""
    monkeypatch.setattr(schemes, "reaction", _planted("schnak_no_gamma"))
    with pytest.raises(AssertionError):
        test_schnakenberg_turing_mode_grows_at_predicted_rate()
