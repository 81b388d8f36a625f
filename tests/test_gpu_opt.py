"""GPU cost functions and optimizer (lbm_opt_cost, lbm_opt_minimize) against
the modified-equation oracle and the paper's Tables 1-3 (sections 3.2, 4.2).
"""
import numpy as np
import pytest

import lbm_inputs as inp
from oracle import modified as md

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1107_4543_gb300 import build, lbm

    build.build()
    lbm.load()
    return lbm


def sig_of(t):
    return (t["sigma_e"], t["sigma_eps"], t["sigma_q"], t["sigma_nu"])


CASES = [("F", 5, "odd", None, False), ("F", 5, "even", None, False), ("F", 5, "all", None, False),
         ("F", 3, "all", None, False), ("F", 6, "odd", None, False),
         ("G", 4, "all", "euler", False), ("G", 4, "all", "ns-bulk", False),
         ("G", 5, "odd", "ns", False), ("G", 4, "even", "euler", True)]


@pytest.mark.parametrize("kind,order,part,ref,fixed", CASES)
def test_cost_matches_oracle(L, kind, order, part, ref, fixed):
    rng = np.random.default_rng(order * 7 + len(part))
    sig = np.column_stack([10 ** rng.uniform(-5, -1, 5), 10 ** rng.uniform(-4, 0.5, 5),
                           10 ** rng.uniform(-4, 2, 5), 10 ** rng.uniform(-5, -1, 5)])
    spec = L.cost_spec(kind, order, part, ref, 0.2 if not fixed else 0.1, fixed)
    got = L.lbm_opt_cost(spec, sig)
    for k in range(len(sig)):
        want = md.cost(sig[k], order, kind, part, 0.2 if not fixed else 0.1, ref,
                       fixed_speed=fixed)
        assert got[k] == pytest.approx(want, rel=1e-11, abs=1e-300), (k, sig[k])
    again = L.lbm_opt_cost(spec, sig)
    assert np.array_equal(got, again)  # fixed reduction order


def test_cost_reproduces_printed_values(L):
    """Appendix D's F^o at two points and the costs of Tables 1-3 at their
    printed optima."""
    f = L.cost_spec("F", 5, "odd")
    assert L.lbm_opt_cost(f, [(0.0025, 0.0, 0.0, 0.0025)])[0] == pytest.approx(57.80191535,
                                                                              rel=2e-9)
    assert L.lbm_opt_cost(f, [sig_of(inp.TABLE1["A"])])[0] == pytest.approx(17.9024342612509066,
                                                                           rel=5e-9)
    g2 = L.cost_spec("G", 4, "all", "euler")
    g3 = L.cost_spec("G", 4, "all", "ns-bulk")
    assert L.lbm_opt_cost(g2, [sig_of(inp.TABLE2["A"])])[0] == pytest.approx(
        14.4537555316616474, rel=2e-9)
    assert L.lbm_opt_cost(g3, [sig_of(inp.TABLE3["B"])])[0] == pytest.approx(
        14.45351071030945, rel=2e-9)


BOUNDS_LO = dict(sigma_eps=0.0, sigma_q=0.0)


@pytest.mark.parametrize("group,part", [("A", "odd"), ("B", "all"), ("C", "odd"), ("D", "all")])
def test_minimizer_reproduces_table1(L, group, part):
    t = inp.TABLE1_READ[group]
    spec = L.cost_spec("F", 5, part)
    r, c, ev = L.lbm_opt_minimize(spec, dict(t, sigma_eps=0.3, sigma_q=1.0),
                                  ("sigma_eps", "sigma_q"), BOUNDS_LO,
                                  dict(sigma_eps=10.0, sigma_q=1000.0))
    assert r["sigma_eps"] <= 1e-9
    assert r["sigma_q"] == pytest.approx(t["sigma_q"], rel=2e-6)
    assert c <= md.cost(sig_of(t), 5, "F", part) * (1 + 1e-12)
    assert ev > 100


# Table 3 group B (sigma_e = 2.5e-6, sigma_nu = 1e-5) has a cost surface so
# flat that 1e-3 in sigma_eps moves G by under 1e-15 relative, below FP64
# resolution: its printed optimum is matched to 2e-2 (and the cost must not
# exceed the printed optimum's), the others to 1e-4.
@pytest.mark.parametrize("table,group,ref,tol", [(2, "A", "euler", 1e-4), (2, "B", "euler", 1e-4),
                                                 (3, "A", "ns-bulk", 1e-4),
                                                 (3, "B", "ns-bulk", 2e-2)])
def test_minimizer_reproduces_tables23(L, table, group, ref, tol):
    t = (inp.TABLE2 if table == 2 else inp.TABLE3)[group]
    spec = L.cost_spec("G", 4, "all", ref)
    hi = dict(sigma_eps=1.0, sigma_q=1.0)
    r, c, _ = L.lbm_opt_minimize(spec, dict(t, sigma_eps=0.5, sigma_q=0.5),
                                 ("sigma_eps", "sigma_q"), BOUNDS_LO, hi)
    assert r["sigma_eps"] == pytest.approx(t["sigma_eps"], rel=tol)
    assert r["sigma_q"] == pytest.approx(t["sigma_q"], rel=tol)
    assert c <= md.cost(sig_of(t), 4, "G", "all", 0.2, ref) * (1 + 1e-12)


def test_invalid_cost_arguments(L):
    with pytest.raises(L.LbmError):
        L.lbm_opt_cost(L.cost_spec("F", 7, "all"), [(0.1, 0.1, 0.1, 0.1)])
    with pytest.raises(L.LbmError):
        L.lbm_opt_cost(L.cost_spec("F", 5, "all"), [(0.1, -0.1, 0.1, 0.1)])
    with pytest.raises(L.LbmError):
        L.lbm_opt_cost(L.cost_spec("G", 4, "all", u0=float("nan")), [(0.1, 0.1, 0.1, 0.1)])
    with pytest.raises(L.LbmError):
        L.lbm_opt_minimize(L.cost_spec("F", 5, "all"), dict(sigma_e=0.1, sigma_eps=0.1,
                                                           sigma_q=0.1, sigma_nu=0.1),
                           ("sigma_q",), dict(sigma_q=1.0), dict(sigma_q=0.5))
