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


def test_row_matches_the_printed_langevin_predictions():
    """At the paper's particle density rho_p = 2 rho_tot, with F_p from
    Eq. (fp) and m_p = pi d^3 rho_p / 6, the row's predictions equal the
    closed forms printed in Section 3: Delta U = sqrt(6 / (pi rho_p L^3))
    (kT)^(1/2) (d/L)^(-3/2) (Eq. (FLUCTUATIONSSCALING)) and Delta U / U =
    18 sqrt(6 eta^2 / (rho_tot^2 pi rho_p L^7)) (kT)^(1/2) (d/L)^(-7/2) / (g c_m)
    (Eq. (normalizedconf)), the unconfined one with c_m = 1."""
    from paper_1909_01092_gb300 import workloads as W

    p = W.params(lx=32, ly=32, lz=64, radius=4.0, rho_p_ratio=2.0, g=5e-6, kT=1e-5, tau_s=0.9)
    rho = p["rho_a0"] + p["rho_b0"]
    rho_p, d, L, kT, g = 2.0 * rho, 8.0, 32.0, 1e-5, 5e-6
    mp = np.pi * d ** 3 / 6 * rho_p
    Fp = np.pi * d ** 3 / 6 * (rho_p - rho) * g
    eta = rho * (0.9 - 0.5) / 3
    U0 = Fp / (3 * np.pi * eta * d)
    rng = np.random.default_rng(5)
    ufl = -1e-6
    vz = ufl + 0.6 * U0 + 1e-4 * rng.standard_normal(5000)
    row = sweep.settling_row(p, vz, ufl, mp, Fp)
    assert row["cm"] == pytest.approx(0.6, abs=5 * 1e-4 / np.sqrt(5000) / U0)
    assert row["dU"] == pytest.approx(1e-4, rel=0.05)
    assert row["dU_pred"] == pytest.approx(np.sqrt(6 / (np.pi * rho_p * L ** 3)) * kT ** 0.5 * (d / L) ** -1.5)
    printed = 18 * np.sqrt(6 * eta ** 2 / (rho ** 2 * np.pi * rho_p * L ** 7)) * kT ** 0.5 * (d / L) ** -3.5 / g
    assert row["dU_over_U_pred"] == pytest.approx(printed / row["cm"])
    assert row["dU0_over_U0_pred"] == pytest.approx(printed)
