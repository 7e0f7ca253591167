"""The m-strategy sweep tool's host side: the strategies follow Tab. 2's layout (Lloyd, then fixed
and dynamic m for each m value, the paper's m-bar = 30) and the table shows accepted / total."""
from paper_1805_10638_gb300 import sweep


def test_tab2_strategies():
    names = [n for n, _ in sweep.tab2_strategies((2, 5))]
    assert names == ["Lloyd", "fixed m=2", "dynamic m0=2", "fixed m=5", "dynamic m0=5"]
    p = dict(sweep.tab2_strategies((3,), m_max=12))
    assert p["Lloyd"] == dict(lloyd_only=1)
    assert p["fixed m=3"] == dict(m_init=3, m_max=12, fixed_m=1)
    assert p["dynamic m0=3"] == dict(m_init=3, m_max=12)
    assert sweep.PAPER_M_MAX == 30


def test_eps_strategies_vary_one_threshold_at_a_time():
    ps = [p for _, p in sweep.eps_strategies()]
    assert ps[0]["eps1"] == 0.02 and ps[0]["eps2"] == 0.5
    for p in ps[1:]:
        assert (p["eps1"] == 0.02) != (p["eps2"] == 0.5)
    assert all(p["m_init"] == 2 and p["m_max"] == 30 for p in ps)


def test_format_table():
    rows = [dict(strategy="fixed m=2", accepted=227, iters=372, ms_per_solve=14.667, mse=8.94807,
                 m_final_mean=2.0)]
    t = sweep.format_table(rows).splitlines()
    assert t[0].startswith("| strategy | #Iter (accepted / total)")
    assert t[2] == "| fixed m=2 | 227 / 372 | 14.67 | 8.94807 | 2.0 |"
