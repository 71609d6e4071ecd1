"""Host check of the settling statistics (paper_1909_01092_gb300.sweep):
five-interval means and fluctuations with their error bars, as the paper's
Section 3 figures define them."""
import numpy as np
import pytest

from paper_1909_01092_gb300 import sweep


def test_interval_statistics_of_a_constructed_series():
    # five intervals of 4 samples: means 1..5, each interval +-d about its mean
    d = np.array([0.1, 0.2, 0.3, 0.4, 0.5])
    v = np.concatenate([[m - s, m + s, m - s, m + s] for m, s in zip([1.0, 2.0, 3.0, 4.0, 5.0], d)])
    st = sweep.interval_stats(v)
    assert st["mean"] == pytest.approx(3.0)
    assert st["mean_err"] == pytest.approx(np.std([1, 2, 3, 4, 5]))
    assert st["fluct"] == pytest.approx(d.mean())
    assert st["fluct_err"] == pytest.approx(d.std())


def test_gaussian_series_recovers_its_parameters():
    rng = np.random.default_rng(3)
    v = 0.25 + 0.01 * rng.standard_normal(50000)
    st = sweep.interval_stats(v)
    assert abs(st["mean"] - 0.25) < 3 * 0.01 / np.sqrt(50000)
    assert abs(st["fluct"] - 0.01) < 1e-4
    assert st["mean_err"] < 1e-3 and st["fluct_err"] < 1e-3


def test_too_short_a_series_is_refused():
    with pytest.raises(ValueError):
        sweep.interval_stats(np.ones(9))


def test_command_line_builds_the_channel_set(monkeypatch, capsys):
    """The command line makes L x L x 2L channels (walls on x and y, the
    counterforce on), `realisations` noise realisations per channel with
    distinct replica indices, and prints one JSON line per replica."""
    seen = {}

    def fake(plist, burn, samples, every=10, intervals=5):
        seen.update(plist=plist, burn=burn, samples=samples, every=every)
        return [{"L": p["lx"], "replica": p["replica"]} for p in plist]

    monkeypatch.setattr(sweep, "settling_sweep", fake)
    sweep.main(["--L", "16", "32", "--radius", "4", "--kT", "1e-5", "--g", "1e-4", "--realisations", "3",
                "--burn", "100", "--samples", "20", "--every", "5"])
    plist = seen["plist"]
    assert [p["lx"] for p in plist] == [16, 16, 16, 32, 32, 32]
    assert all(p["lz"] == 2 * p["lx"] and p["ly"] == p["lx"] for p in plist)
    assert all(p["wall"] == (1, 1, 0) and p["fluid_counterforce"] == 1 for p in plist)
    assert len({p["replica"] for p in plist}) == 6
    assert all(p["radius"] == 4.0 and p["kT"] == 1e-5 and p["g"] == 1e-4 for p in plist)
    assert (seen["burn"], seen["samples"], seen["every"]) == (100, 20, 5)
    assert len(capsys.readouterr().out.strip().splitlines()) == 6
