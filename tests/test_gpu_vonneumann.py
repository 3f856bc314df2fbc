"""The von Neumann tool (fdlbm_vn_spectrum, Sec. 4, Eqs. 18-20) on the GPU against the oracle.

- The matrix G equals the oracle's element by element. Against the FP64 oracle (pinned by the
  linearised step) the bound is 1e-10 of max|G|, the accuracy of its numerical derivatives.
  Against the 40-digit oracle it is 1e-14 of max|G|, including at the Fig. 2 state.
- The 33 eigenvalues equal the 40-digit oracle's to 1e-12, and max|omega| to 1e-12, at states
  where FP64 eigenvalues are wrong by up to 0.05.
- At zero wave number the spectrum is {1 (x4), 1 - dt/tau (x29)} (J is a projector).
- Over many well-conditioned random cases max|omega| agrees with FP64 LAPACK eigenvalues of the
  FP64 oracle matrix to 1e-9.
- Invalid cases are flagged, not computed.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import vonneumann as V  # noqa: E402
from paper_0801_4169_gb300 import fdlbm as F  # noqa: E402

DPS = 40


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    F.lib()


def _match(a, b):
    a = list(a)
    err = 0.0
    for z in b:
        j = int(np.argmin([abs(z - w) for w in a]))
        err = max(err, abs(z - a[j]))
        a.pop(j)
    return err


def _mp_to_np(G):
    return np.array([[complex(G[i, j]) for j in range(33)] for i in range(33)])


HARD = [  # (state, xi_x, xi_y, dx, dy, dt, tau, lambda)
    ((2.0, 30.0, 0.0, 1.0), 0.3, 0.0, 3e-3, 3e-3, 1e-5, 1e-5, 0.5),     # Fig. 2 state
    ((2.0, 30.0, 0.0, 1.0), 1.5, 0.0, 3e-3, 3e-3, 1e-5, 1e-5, 0.0),
    ((2.0, 5.0, 2.0, 25.0), 0.7, 1.9, 3e-3, 3e-3, 1e-5, 1e-5, 0.5),      # Fig. 5 range
    ((50.0 / 17.0, 16.7, -5.71578, 22.61), 2.0, -0.4, 3e-3, 3e-3, 1e-5, 2e-5, 1.0),  # Sec. 5.2 top state
    ((1.0, 0.5, -0.3, 0.8), np.pi, 1.1, 1e-3, 2e-3, 1e-5, 1e-4, 2.0),
]


@pytest.mark.parametrize("case", HARD)
def test_matrix_and_spectrum_match_the_high_precision_oracle(case):
    st, xx, xy, dx, dy, dt, tau, lam = case
    c = F.vn_cases([st], xx, xy, lam)
    mx, status, om, G = F.vn_spectrum(c, dx, dy, dt, tau, eigenvalues=True, matrix=True)
    assert status[0] == F.FDLBM_VN_OK
    Gm = V.amplification_matrix_mp(st, xx, xy, dx, dy, dt, tau, lam, dps=DPS)
    Gref = _mp_to_np(Gm)
    assert np.max(np.abs(G[0] - Gref)) <= 1e-14 * np.abs(Gref).max()
    ev = [complex(z) for z in V.eigvals_mp(Gm, DPS)]
    assert _match(om[0], ev) <= 1e-12
    assert abs(mx[0] - max(abs(z) for z in ev)) <= 1e-12


@pytest.mark.parametrize("xi", [(0.3, 0.0), (2.0, -0.4), (np.pi, 1.1)])
def test_matrix_matches_the_fp64_oracle(xi):
    st, args = (1.0, 0.3, -0.2, 1.0), (3e-3, 2e-3, 1e-5, 2e-5)
    for flags, kw in ((0, {}), (F.FDLBM_NO_LW, dict(lw=False)), (F.FDLBM_NO_DISP, dict(disp=False)),
                      (F.FDLBM_NO_VISC, dict(visc=False))):
        _, status, _, G = F.vn_spectrum(F.vn_cases([st], xi[0], xi[1], 0.5, flags), *args, matrix=True)
        ref = V.amplification_matrix(st, xi[0], xi[1], *args, 0.5, **kw)
        assert status[0] == 0 and np.max(np.abs(G[0] - ref)) <= 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("st,tau", [((2.0, 30.0, 0.0, 1.0), 1e-5), ((1.0, 0.5, -0.3, 0.8), 1e-4)])
def test_zero_wavenumber_spectrum_is_that_of_a_projector(st, tau):
    dt = 1e-5
    _, status, om, _ = F.vn_spectrum(F.vn_cases([st], 0.0, 0.0, 0.5), 3e-3, 3e-3, dt, tau, eigenvalues=True)
    z = om[0]
    ones = np.abs(z - 1.0) < 1e-8
    assert status[0] == 0 and ones.sum() == 4
    assert np.max(np.abs(z[ones] - 1.0)) <= 1e-13 and np.max(np.abs(z[~ones] - (1.0 - dt / tau))) <= 1e-13


def test_many_well_conditioned_cases_match_fp64_lapack():
    rng = np.random.default_rng(3)
    n = 256
    st = np.stack([rng.uniform(0.5, 2.0, n), rng.uniform(-1.5, 1.5, n), rng.uniform(-1.5, 1.5, n),
                   rng.uniform(0.6, 1.5, n)], axis=1)
    xx, xy, lam = rng.uniform(-np.pi, np.pi, n), rng.uniform(-np.pi, np.pi, n), rng.uniform(0, 3, n)
    flags = rng.integers(0, 8, n)
    c = F.vn_cases(st, xx, xy, lam, flags)
    args = (2e-3, 3e-3, 1e-5, 2e-5)
    mx, status, om, _ = F.vn_spectrum(c, *args, eigenvalues=True)
    assert np.all(status == 0)
    for k in range(0, n, 8):
        G = V.amplification_matrix(tuple(st[k]), xx[k], xy[k], *args, lam[k], lw=not flags[k] & 1,
                                   disp=not flags[k] & 2, visc=not flags[k] & 4)
        ev = np.linalg.eigvals(G)
        assert abs(mx[k] - np.abs(ev).max()) <= 1e-9
        assert _match(om[k], ev) <= 1e-8


def test_invalid_cases_are_flagged():
    c = F.vn_cases([(1.0, 0.0, 0.0, 1.0), (0.0, 0.0, 0.0, 1.0), (1.0, 0.0, 0.0, -1.0), (1.0, np.nan, 0.0, 1.0),
                    (1.0, 0.0, 0.0, 1.0), (1.0, 0.0, 0.0, 1.0)], [0.5, 0.5, 0.5, 0.5, 9.0, 0.5], 0.0,
                   [0.5, 0.5, 0.5, 0.5, 0.5, -1.0])
    mx, status, om, _ = F.vn_spectrum(c, 1e-3, 1e-3, 1e-5, 1e-5, eigenvalues=True)
    assert list(status) == [0, 1, 1, 1, 1, 1]
    assert np.isfinite(mx[0]) and np.all(np.isnan(mx[1:])) and np.all(np.isnan(om[1:]))


def test_sec4_claims_hold_at_the_papers_states():
    """Sec. 4 in double-double, at the paper's own states (Figs. 2, 4, 5, 6; 128 wave numbers):
    - Fig. 2: line II (Lax-Wendroff) lowers max|omega| and line III (dispersion) raises it;
    - Fig. 4: max|omega| falls with lambda, above 1 for lambda <= 0.1, below 1 for lambda >= 1;
    - Fig. 5: it falls as T grows; Fig. 6: it grows with u1.
    Two of the maxima are checked against the 40-digit oracle at their wave number."""
    from paper_0801_4169_gb300 import workloads as W
    rows, curves, xi = W.vn_sec4_cases(nk=128)
    cases = F.vn_cases(rows[:, :4], rows[:, 4], rows[:, 5], rows[:, 6], rows[:, 7].astype(np.int32))
    dx, dy, dt, tau = W.VN_SEC4_GRID
    mx, status, _, _ = F.vn_spectrum(cases, dx, dy, dt, tau)
    assert np.all(status == 0)
    mx = mx.reshape(len(curves), len(xi))
    peak = {c[0]: float(mx[k].max()) for k, c in enumerate(curves)}
    arg = {c[0]: float(xi[int(mx[k].argmax())]) for k, c in enumerate(curves)}
    assert peak["fig2 lines I-II"] < peak["fig2 line I"] < peak["fig2 lines I,III"]
    lams = [peak["fig4 lambda=%g" % l] for l in (0.05, 0.1, 0.5, 1.0, 1.8, 2.0, 3.0)]
    assert all(b < a for a, b in zip(lams, lams[1:])) and lams[1] > 1.0 and max(lams[3:]) < 1.0
    Ts = [peak["fig5 T=%g" % T] for T in (1, 5, 15, 25)]
    assert all(b < a for a, b in zip(Ts, Ts[1:]))
    us = [peak["fig6 u1=%g" % u] for u in (0, 5, 10, 15, 20, 25, 30)]
    assert us[1] >= us[0] - 1e-12 and all(b > a for a, b in zip(us[1:], us[2:]))
    for name, st, lam, fl in (("fig2 all", (2.0, 30.0, 0.0, 1.0), 0.5, 0), ("fig6 u1=30", (2.0, 30.0, 0.0, 1.0), 0.0, 0)):
        ref = V.max_abs_eig_mp(st, arg[name], 0.0, dx, dy, dt, tau, lam, dps=DPS)
        assert abs(peak[name] - ref) <= 1e-12
