"""The oracle's OpenMP collision loop writes each node's populations from
that node's inputs only, so its results do not depend on the thread count:
one thread and all threads give bit-identical fields and particle records,
here on the fluctuating channel with a moving, wetted sphere."""
import numpy as np

from paper_1909_01092_gb300 import workloads as W


def test_results_do_not_depend_on_the_thread_count(oracle_mod):
    p = W.channel_small(kT=1e-5, delta_rho=0.3, G=1.2)
    full = oracle_mod.num_threads()
    out = []
    try:
        for threads in (1, max(full, 2)):
            oracle_mod.set_threads(threads)
            o = oracle_mod.Oracle(p)
            o.set_particle(p["pos0"], V=(0.01, -0.005, 0.03), Omega=(0.001, 0.0, -0.002))
            o.step(12)
            out.append((o.get_f(), o.particle()))
    finally:
        oracle_mod.set_threads(full)
    (f1, p1), (f2, p2) = out
    assert np.array_equal(f1, f2)
    for key in ("X", "V", "Omega", "F", "T"):
        assert np.array_equal(p1[key], p2[key]), key
    assert p1["nfluid"] == p2["nfluid"]
