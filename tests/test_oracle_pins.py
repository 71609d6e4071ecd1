"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: published
known-answer vectors, closed forms of the lattice and of the Shan-Chen force,
exact invariants of the scheme, and transport coefficients printed in the paper
(eta = 0.383 and D = 1/6 at tau = 1, Section 2). A dropped term, a wrong sign,
a wrong weight or a transposed operand in the oracle fails one of them.
"""
import math
import os

import numpy as np
import pytest

from paper_1909_01092_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# Printed D3Q19 velocity set in the documented direction order.
C = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
              [1, 1, 0], [-1, -1, 0], [1, -1, 0], [-1, 1, 0], [1, 0, 1], [-1, 0, -1], [1, 0, -1],
              [-1, 0, 1], [0, 1, 1], [0, -1, -1], [0, 1, -1], [0, -1, 1]], dtype=float)


def _feq(rho, u):
    """Textbook second-order equilibrium, written from the lattice tables."""
    w = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
    cu = C @ u
    return w * rho * (1 + 3 * cu + 4.5 * cu ** 2 - 1.5 * (u @ u))


# ---------------------------------------------------------------------------
# Philox4x32-10 and the normal deviates
# ---------------------------------------------------------------------------
def test_philox_known_answer_vectors(oracle_mod):
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if ln.strip() and ln[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = oracle_mod.philox(v[0:4], v[4:6])
        assert list(out) == v[6:10]


def test_uniform_map_is_open_and_exact_in_binary32(oracle_mod):
    lo, hi = oracle_mod.uniform(0), oracle_mod.uniform(0xFFFFFFFF)
    assert lo == 0.5 * 2.0 ** -23 and hi == 1.0 - 0.5 * 2.0 ** -23
    for x in (0, 1, 511, 512, 12345678, 0x80000000, 0xFFFFFFFF):
        u = oracle_mod.uniform(x)
        assert 0.0 < u < 1.0
        assert float(np.float32(u)) == u


def test_normals_are_standard_gaussian(oracle_mod):
    from scipy import stats
    z = np.concatenate([oracle_mod.normals(99, 3, 7, n) for n in range(4000)])
    assert abs(z.mean()) < 4 / math.sqrt(z.size)
    assert abs(z.var() - 1) < 4 * math.sqrt(2 / z.size)
    assert stats.kstest(z, "norm").pvalue > 1e-3
    zz = z.reshape(4000, 36)
    corr = np.corrcoef(zz.T) - np.eye(36)
    assert np.abs(corr).max() < 5 / math.sqrt(4000)


def test_normals_depend_on_every_key_field(oracle_mod):
    base = oracle_mod.normals(5, 0, 0, 0)
    for args in ((6, 0, 0, 0), (5, 1, 0, 0), (5, 0, 1, 0), (5, 0, 0, 1), (5 + (1 << 32), 0, 0, 0)):
        assert not np.allclose(oracle_mod.normals(*args), base)


# ---------------------------------------------------------------------------
# Lattice and mode basis (D3Q19, Section 2)
# ---------------------------------------------------------------------------
def test_lattice_isotropy(oracle_mod):
    L = oracle_mod.lattice()
    c, w, opp = L["c"], L["w"], L["opp"]
    assert np.array_equal(c, C)
    assert abs(w.sum() - 1) < 1e-15
    assert np.abs(w @ c).max() < 1e-16
    assert np.allclose(np.einsum("i,ia,ib->ab", w, c, c), np.eye(3) / 3, atol=1e-15)
    d = np.eye(3)
    iso4 = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d) + np.einsum("ad,bc->abcd", d, d)) / 9
    assert np.allclose(np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c), iso4, atol=1e-15)
    assert np.array_equal(c[opp], -c)


def test_mode_basis_orthogonal_with_closed_form_norms(oracle_mod):
    L = oracle_mod.lattice()
    e, w, b = L["e"], L["w"], L["b"]
    gram = (e * w) @ e.T
    assert np.allclose(gram, np.diag(b), atol=1e-15)
    expect = [1, 1 / 3, 1 / 3, 1 / 3, 2 / 3, 4 / 3, 4 / 9, 1 / 9, 1 / 9, 1 / 9,
              2 / 3, 2 / 3, 2 / 3, 2 / 9, 2 / 9, 2 / 9, 2, 4 / 3, 4 / 9]
    assert np.allclose(b, expect, atol=1e-15)
    # rows 0..3 are density and momentum
    assert np.array_equal(e[0], np.ones(19))
    assert np.array_equal(e[1:4], C.T)


# ---------------------------------------------------------------------------
# Collision: equilibrium, forcing, rest state (Eq. lbe, MRT, Section 2)
# ---------------------------------------------------------------------------
def test_single_node_collision_is_second_order_equilibrium(oracle_mod):
    """On a 1x1x1 periodic lattice streaming is the identity, so one step with
    tau = 1 returns f_eq(rho_l, u) of the textbook polynomial, u = sum_l j_l / rho_tot."""
    p = W.params(lx=1, ly=1, lz=1, wall=(0, 0, 0), G=1.5)
    o = oracle_mod.Oracle(p)
    rng = np.random.default_rng(3)
    f = rng.uniform(0.01, 0.1, size=(2, 19, 1, 1, 1))
    o.set_f(f)
    o.step(1)
    out = o.get_f()[:, :, 0, 0, 0]
    rho = f[:, :, 0, 0, 0].sum(1)
    j = (f[:, :, 0, 0, 0] @ C).sum(0)
    u = j / rho.sum()
    for l in range(2):
        assert np.allclose(out[l], _feq(rho[l], u), rtol=1e-13, atol=1e-16)


def test_single_node_forcing_matches_guo_source(oracle_mod):
    """With a body force F_l the tau = 1 result is f_eq(rho_l, u) + 1/2 S_i, where S_i
    is the second-order (Guo-type) source w_i [3 (c - u).F + 9 (c.u)(c.F)] and
    u = (j + F/2) / rho_tot (the hydrodynamical velocity v^(H) of Section 2)."""
    g = np.array([1e-3, -2e-3, 3e-3])
    p = W.params(lx=1, ly=1, lz=1, wall=(0, 0, 0), fluid_force=tuple(g))
    o = oracle_mod.Oracle(p)
    rng = np.random.default_rng(4)
    f = rng.uniform(0.01, 0.1, size=(2, 19, 1, 1, 1))
    o.set_f(f)
    o.step(1)
    out = o.get_f()[:, :, 0, 0, 0]
    f0 = f[:, :, 0, 0, 0]
    rho = f0.sum(1)
    Fl = np.outer(rho / rho.sum(), g)
    u = ((f0 @ C).sum(0) + 0.5 * Fl.sum(0)) / rho.sum()
    w = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
    for l in range(2):
        S = w * (3 * (C - u) @ Fl[l] + 9 * (C @ u) * (C @ Fl[l]))
        assert np.allclose(out[l], _feq(rho[l], u) + 0.5 * S, rtol=1e-13, atol=1e-16)


def test_uniform_rest_state_is_fixed_point_with_walls(oracle_mod):
    p = W.params(lx=6, ly=5, lz=4, wall=(1, 1, 0), G=1.2, init_pert=0.0)
    o = oracle_mod.Oracle(p)
    f0 = o.get_f()
    o.step(10)
    assert np.allclose(o.get_f(), f0, rtol=0, atol=1e-15)


@pytest.mark.parametrize("i", range(1, 19))
def test_free_streaming_and_halfway_walls(oracle_mod, i):
    """With every relaxation time infinite (no collision), G = 0 and no noise,
    a pulse moves one node per step along c_i; at a wall it comes back on the
    opposite direction one step later (halfway bounce-back)."""
    inf = float("inf")
    p = W.params(lx=4, ly=4, lz=4, wall=(1, 1, 0), tau_s=inf, tau_d=inf, tau_g=inf, G=0.0, init_pert=0.0)
    o = oracle_mod.Oracle(p)
    base = o.get_f()
    f = base.copy()
    x0 = np.array([1, 2, 1])
    f[0, i, x0[2], x0[1], x0[0]] += 0.25
    o.set_f(f)
    opp = [0, 2, 1, 4, 3, 6, 5, 8, 7, 10, 9, 12, 11, 14, 13, 16, 15, 18, 17]
    pos, d = x0.copy(), i
    for _ in range(6):
        o.step(1)
        nxt = pos + C[d].astype(int)
        if nxt[0] < 0 or nxt[0] > 3 or nxt[1] < 0 or nxt[1] > 3:
            d = opp[d]
        else:
            pos = nxt
            pos[2] %= 4
        g = o.get_f() - base
        want = np.zeros_like(g)
        want[0, d, pos[2], pos[1], pos[0]] = 0.25
        assert np.allclose(g, want, atol=1e-14)


# ---------------------------------------------------------------------------
# Shan-Chen force, Eq. (sc-force), with omega_i = D3Q19 weights
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_sc_force_on_a_sine_wave(oracle_mod, axis):
    """rho_B = rho_B0 (1 + a sin(k x_axis)), rho_A uniform. Summing Eq. (sc-force)
    by hand with the D3Q19 weights (1/6 of the weight on each side of the axis):
    F_A = -G rho_A rho_B0 a sin(k) cos(k x) / 3 along the axis, F_B = 0."""
    L, G, a = 12, 1.3, 0.1
    dims = [1, 1, 1]
    dims[axis] = L
    p = W.params(lx=dims[0], ly=dims[1], lz=dims[2], wall=(0, 0, 0), G=G, init_pert=0.0)
    o = oracle_mod.Oracle(p)
    f = o.get_f()
    k = 2 * np.pi / L
    s = np.arange(L)
    prof = (1 + a * np.sin(k * s)).reshape([L if ax == axis else 1 for ax in (2, 1, 0)])
    f[1] = f[1] * prof[None]
    o.set_f(f)
    fl = o.fields()
    rhoA = p["rho_a0"]
    want = -G * rhoA * p["rho_b0"] * a * np.sin(k) * np.cos(k * s) / 3
    got = fl["force"][0, axis].reshape(L)
    assert np.allclose(got, want, rtol=1e-12, atol=1e-17)
    for ax in range(3):
        if ax != axis:
            assert np.abs(fl["force"][0, ax]).max() < 1e-17
    assert np.abs(fl["force"][1]).max() < 1e-17


@pytest.mark.parametrize("drho", [0.0, 0.02, 0.5, -0.3])
def test_virtual_layer_and_sc_reaction(oracle_mod, drho):
    """A sphere at rest in a uniform mixture (Section 2: virtual fluid layer).
    Surface particle nodes carry psi = (rho_A + drho, rho_B - drho), clipped at 0;
    nodes with no fluid neighbour carry 0. The force on a fluid node next to the
    sphere is -G rho_l sum over its particle-node directions of w_i (psi_l'(s) - rho_l') c_i,
    and the reaction on the particle is minus the sum of those forces."""
    G = 1.2
    p = W.params(lx=12, ly=12, lz=12, wall=(0, 0, 0), G=G, init_pert=0.0, radius=3.3, delta_rho=drho,
                 pos0=(5.3, 5.6, 5.9))
    o = oracle_mod.Oracle(p)
    fl = o.fields()
    ra, rb = p["rho_a0"], p["rho_b0"]
    X = np.array(p["pos0"])
    zz, yy, xx = np.meshgrid(np.arange(12), np.arange(12), np.arange(12), indexing="ij")
    pts = np.stack([xx, yy, zz], -1).astype(float)
    d = pts - X
    d -= 12 * np.floor(d / 12 + 0.5)
    solid = (d ** 2).sum(-1) < 3.3 ** 2
    assert np.array_equal(fl["solid"], solid)
    va, vb = max(ra + drho, 0.0), max(rb - drho, 0.0)
    w = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
    tot = np.zeros(3)
    for z in range(12):
        for y in range(12):
            for x in range(12):
                nb = [((x + int(c[0])) % 12, (y + int(c[1])) % 12, (z + int(c[2])) % 12) for c in C[1:]]
                if solid[z, y, x]:
                    has_fluid = any(not solid[q[2], q[1], q[0]] for q in nb)
                    want = (va, vb) if has_fluid else (0.0, 0.0)
                    assert np.allclose(fl["psi"][:, z, y, x], want, atol=1e-15)
                    continue
                fa = np.zeros(3)
                fb = np.zeros(3)
                for idx, q in enumerate(nb, start=1):
                    if solid[q[2], q[1], q[0]]:
                        fa += -G * ra * w[idx] * (vb - rb) * C[idx]
                        fb += -G * rb * w[idx] * (va - ra) * C[idx]
                assert np.allclose(fl["force"][0, :, z, y, x], fa, atol=1e-15)
                assert np.allclose(fl["force"][1, :, z, y, x], fb, atol=1e-15)
                tot += fa + fb
    assert np.allclose(fl["sc_reaction_force"], -tot, atol=1e-13)


def test_neutral_wall_ghosts_exert_no_force_on_uniform_fluid(oracle_mod):
    p = W.params(lx=5, ly=6, lz=3, wall=(1, 1, 1), G=1.5, init_pert=0.0)
    o = oracle_mod.Oracle(p)
    assert np.abs(o.fields()["force"]).max() < 1e-16


def test_wall_ghost_is_mean_of_fluid_neighbours(oracle_mod):
    """rho_B varies along y; walls on x. A node at x = 0 sees, across the wall,
    ghosts whose psi is the mean over their fluid neighbours (Delta rho = 0)."""
    G = 1.0
    p = W.params(lx=3, ly=6, lz=1, wall=(1, 0, 0), G=G, init_pert=0.0)
    o = oracle_mod.Oracle(p)
    f = o.get_f()
    prof = np.array([1.0, 1.3, 0.7, 1.1, 0.9, 1.2])
    f[1] *= prof[None, None, :, None]
    o.set_f(f)
    fl = o.fields()
    rb = p["rho_b0"] * prof
    ra = p["rho_a0"]
    w = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
    # ghost at (-1, y): fluid neighbours (0, y), (0, y+-1) (z is a single periodic layer,
    # so (0, y, z+-1) is (0, y) again twice)
    def ghost(y):
        vals = [rb[y], rb[(y + 1) % 6], rb[(y - 1) % 6], rb[y], rb[y]]
        return np.mean(vals)
    x, y = 0, 2
    acc = np.zeros(3)
    for i in range(1, 19):
        cx, cy, cz = C[i].astype(int)
        nx, ny = x + cx, (y + cy) % 6
        psi = ghost(ny) if nx < 0 else rb[ny]
        acc += w[i] * psi * C[i]
    assert np.allclose(fl["force"][0, :, 0, y, x], -G * ra * acc, atol=1e-15)


# ---------------------------------------------------------------------------
# Exact invariants
# ---------------------------------------------------------------------------
def test_mass_and_momentum_conservation_with_noise_and_sc(oracle_mod):
    p = W.params(lx=6, ly=5, lz=7, wall=(0, 0, 0), G=1.5, kT=1e-4, tau_s=0.9, tau_d=1.3, tau_g=0.8)
    o = oracle_mod.Oracle(p)
    o.set_f(W.random_populations(p, 11))
    a = o.observables()
    o.step(15)
    b = o.observables()
    assert np.allclose(b["mass"], a["mass"], rtol=1e-13)
    assert np.allclose(b["momentum"], a["momentum"], rtol=0, atol=1e-12)


def test_constant_force_momentum_growth(oracle_mod):
    """Total momentum grows by exactly N F per step under a constant body force."""
    g = np.array([1e-5, -2e-5, 3e-5])
    p = W.params(lx=4, ly=5, lz=3, wall=(0, 0, 0), G=1.2, kT=1e-5, fluid_force=tuple(g))
    o = oracle_mod.Oracle(p)
    o.set_f(W.random_populations(p, 12))
    a = o.observables()["momentum"]
    o.step(7)
    b = o.observables()["momentum"]
    assert np.allclose(b - a, 7 * 60 * g, rtol=1e-10, atol=1e-14)


def test_particle_closes_mass_and_momentum(oracle_mod):
    """A sphere moving through a periodic box (walls off, no driving force),
    with Shan-Chen forces, wetting and noise: fluid mass plus the pending mass
    correction is conserved per component, and fluid momentum plus particle
    momentum plus the pending cover/uncover impulse is conserved exactly,
    through bounce-back, virtual-layer reactions and cover/uncover events."""
    p = W.params(lx=12, ly=12, lz=12, wall=(0, 0, 0), G=1.2, kT=1e-5, radius=2.7, delta_rho=0.3)
    o = oracle_mod.Oracle(p)
    o.set_particle(p["pos0"], V=(0.05, -0.03, 0.08), Omega=(0.01, 0.0, -0.02))

    def inv():
        ob, pa = o.observables(), o.particle()
        return ob["mass"] + ob["pending_mass"], ob["momentum"] + ob["particle_momentum"] + pa["Ppend"]

    m0, p0 = inv()
    n0 = o.particle()["nfluid"]
    changed = False
    for _ in range(12):
        o.step(1)
        changed |= o.particle()["nfluid"] != n0
        m1, p1 = inv()
        assert np.allclose(m1, m0, rtol=1e-13)
        assert np.allclose(p1, p0, rtol=0, atol=1e-12)
    assert changed  # cover/uncover happened


def test_particle_at_rest_feels_no_force_and_starts_with_fp_over_mp(oracle_mod):
    """A centred sphere at rest in a uniform mixture: the exchanged force is zero
    by symmetry, so after one step V = F_p / m_p along z exactly, with
    F_p = (4/3) pi R^3 (rho_p - rho_tot) g and m_p = (4/3) pi R^3 rho_p (Eq. fp)."""
    R, ratio, g = 3.0, 1.5, 1e-5
    p = W.params(lx=16, ly=16, lz=16, wall=(1, 1, 0), G=1.2, init_pert=0.0, radius=R, rho_p_ratio=ratio, g=g,
                 pos0=(7.5, 7.5, 7.5))
    o = oracle_mod.Oracle(p)
    o.step(1)
    pa = o.particle()
    rt = p["rho_a0"] + p["rho_b0"]
    vol = 4 / 3 * math.pi * R ** 3
    assert math.isclose(pa["Fp"], vol * (ratio * rt - rt) * g, rel_tol=1e-14)
    assert math.isclose(pa["mp"], vol * ratio * rt, rel_tol=1e-14)
    assert np.abs(pa["F"]).max() < 1e-14
    assert np.allclose(pa["V"], [0, 0, pa["Fp"] / pa["mp"]], rtol=1e-12, atol=1e-16)
    assert np.allclose(pa["X"], np.array(p["pos0"]) + pa["V"], rtol=1e-15)


def test_moving_sphere_is_dragged_backwards(oracle_mod):
    p = W.params(lx=14, ly=14, lz=14, wall=(0, 0, 0), G=0.0, init_pert=0.0, radius=3.0)
    o = oracle_mod.Oracle(p)
    V = np.array([0.0, 0.0, 0.01])
    o.set_particle(p["pos0"], V=V)
    o.step(1)
    F = o.particle()["F"]
    assert F[2] < 0 and abs(F[0]) < 1e-3 * abs(F[2]) and abs(F[1]) < 1e-3 * abs(F[2])


# ---------------------------------------------------------------------------
# Transport coefficients printed in the paper (Section 2: eta = 0.383, D = 1/6)
# ---------------------------------------------------------------------------
def _shear_decay_rate(oracle_mod, tau_s, L=48, steps=120):
    p = W.params(lx=L, ly=1, lz=1, wall=(0, 0, 0), G=0.0, tau_s=tau_s, init_pert=0.0, rho_a0=2.21, rho_b0=0.09)
    o = oracle_mod.Oracle(p)
    x = np.arange(L)
    k = 2 * np.pi / L
    A = 1e-4
    f = np.zeros((2, 19, 1, 1, L))
    for l, r in enumerate((2.21, 0.09)):
        for n in range(L):
            f[l, :, 0, 0, n] = _feq(r, np.array([0.0, A * np.sin(k * x[n]), 0.0]))
    o.set_f(f)

    def amp():
        g = o.get_f()
        uy = np.einsum("li...,i->...", g, C[:, 1]).reshape(L) / 2.3
        return 2 * (uy * np.sin(k * x)).mean()

    a0 = amp()
    o.step(steps)
    a1 = amp()
    return -math.log(a1 / a0) / steps / k ** 2


@pytest.mark.parametrize("tau_s", [1.0, 0.8])
def test_shear_wave_gives_printed_viscosity(oracle_mod, tau_s):
    """A decaying shear wave measures the kinematic viscosity nu = (tau - 1/2)/3.
    At tau = 1 and rho_A + rho_B = 2.3 this is eta = rho nu = 0.383 (Section 2)."""
    nu = _shear_decay_rate(oracle_mod, tau_s)
    assert abs(nu - (tau_s - 0.5) / 3) < 0.005 * nu
    if tau_s == 1.0:
        assert abs(2.3 * nu - 0.383) < 0.001


@pytest.mark.parametrize("tau_s,G,rho_a,rho_b", [(0.8, 0.0, 2.21, 0.09), (1.3, 0.0, 2.21, 0.09),
                                               (0.8, 0.5, 1.0, 1.0), (1.3, 0.8, 1.0, 1.0)])
def test_sound_wave_speed_and_damping(oracle_mod, tau_s, G, rho_a, rho_b):
    """The momentum equation of Section 2 has the printed bulk pressure
    P_b = rho_tot / 3 + (G/3) rho_A rho_B and the viscous stress
    eta (grad v + grad v^T), with no separate bulk term. Linearised, a
    standing density wave of wavenumber k at fixed composition then oscillates
    at omega^2 = k^2 dP_b/drho = k^2 [1/3 + (2G/3) rho_A rho_B / rho_tot] (the
    Shan-Chen stencil turning one k of the interaction term into sin k), and
    its amplitude decays at Gamma = nu k^2. The wave runs through the trace and
    normal-stress modes, which a shear wave never touches. In the symmetric
    mixture rho_A = rho_B the wave leaves the composition alone. omega and
    Gamma are the eigenvalue e^(-Gamma +- i omega) of the one-step map of the
    (density, momentum) amplitudes, fitted by least squares once the kinetic
    modes have relaxed."""
    L, eps, steps, skip = 48, 1e-4, 400, 20
    p = W.params(lx=L, ly=1, lz=1, wall=(0, 0, 0), G=G, tau_s=tau_s, init_pert=0.0, rho_a0=rho_a, rho_b0=rho_b)
    o = oracle_mod.Oracle(p)
    k = 2 * np.pi / L
    x = np.arange(L)
    f = np.zeros((2, 19, 1, 1, L))
    for l, r in enumerate((rho_a, rho_b)):
        for n in range(L):
            f[l, :, 0, 0, n] = _feq(r * (1 + eps * np.cos(k * x[n])), np.zeros(3))
    o.set_f(f)
    amps = []
    for _ in range(steps):
        g = o.get_f()
        rho = g.sum((0, 1)).reshape(L)
        jx = np.einsum("li...,i->...", g, C[:, 0]).reshape(L)
        amps.append([2 * ((rho - rho.mean()) * np.cos(k * x)).mean(), 2 * (jx * np.sin(k * x)).mean()])
        o.step(1)
    a = np.array(amps[skip:])
    M = np.linalg.lstsq(a[:-1], a[1:], rcond=None)[0].T
    lam = np.linalg.eigvals(M)[0]
    nu = (tau_s - 0.5) / 3
    omega = math.sqrt(k * k / 3 + (2 * G / 3) * rho_a * rho_b / (rho_a + rho_b) * k * math.sin(k))
    assert abs(-math.log(abs(lam)) / (nu * k * k) - 1) < 0.01
    assert abs(abs(np.angle(lam)) / omega - 1) < 0.003


def test_interdiffusion_gives_printed_diffusivity(oracle_mod):
    """A composition wave at constant total density (G = 0) decays with the
    diffusivity D = (tau_d - 1/2)/3 = 1/6 at tau_d = 1 (Section 2)."""
    L = 48
    p = W.params(lx=L, ly=1, lz=1, wall=(0, 0, 0), G=0.0, init_pert=0.0, rho_a0=1.0, rho_b0=1.0)
    o = oracle_mod.Oracle(p)
    k = 2 * np.pi / L
    x = np.arange(L)
    c = 0.01 * np.sin(k * x)
    f = np.zeros((2, 19, 1, 1, L))
    for n in range(L):
        f[0, :, 0, 0, n] = _feq(1.0 + c[n], np.zeros(3))
        f[1, :, 0, 0, n] = _feq(1.0 - c[n], np.zeros(3))
    o.set_f(f)

    def amp():
        rA = o.get_f()[0].sum(0).reshape(L)
        return 2 * ((rA - 1.0) * np.sin(k * x)).mean()

    a0 = amp()
    o.step(150)
    D = -math.log(amp() / a0) / 150 / k ** 2
    assert abs(D - 1 / 6) < 0.005 / 6


@pytest.mark.parametrize("G,tau_d", [(0.5, 1.0), (0.8, 1.0), (0.8, 0.8)])
def test_shan_chen_interaction_slows_interdiffusion_as_the_chemical_potential_says(oracle_mod, G, tau_d):
    """Section 2: the composition relaxes down the gradient of the chemical
    potential mu = (1/3) ln rho_A - (1/3) ln rho_B - (G/3)(rho_A - rho_B)
    (with the sign that makes the printed coexistence densities equal mu).
    Around a uniform mixture at constant total density, d mu / d rho_A is
    scaled by 1 - 2 G rho_A rho_B / rho_tot when the interaction is on, and
    the mobility in front of grad mu is the same with or without it. So a
    composition wave decays at the G = 0 diffusivity times that factor. The
    Shan-Chen stencil turns the gradient of a wave exp(i k x) into sin(k)
    instead of k, which the factor carries for the force term. The symmetric
    mixture rho_A = rho_B keeps the wave away from pressure, since
    rho_A rho_B is then stationary to first order."""
    L, eps, skip, steps = 96, 1e-4, 50, 300
    k = 2 * np.pi / L
    x = np.arange(L)

    def decay_rate(g):
        p = W.params(lx=L, ly=1, lz=1, wall=(0, 0, 0), G=g, tau_d=tau_d, init_pert=0.0, rho_a0=1.0, rho_b0=1.0)
        o = oracle_mod.Oracle(p)
        c = eps * np.sin(k * x)
        f = np.zeros((2, 19, 1, 1, L))
        for n in range(L):
            f[0, :, 0, 0, n] = _feq(1.0 + c[n], np.zeros(3))
            f[1, :, 0, 0, n] = _feq(1.0 - c[n], np.zeros(3))
        o.set_f(f)

        def amp():
            return 2 * ((o.get_f()[0].sum(0).reshape(L) - 1.0) * np.sin(k * x)).mean()

        o.step(skip)
        a0 = amp()
        o.step(steps)
        return -math.log(amp() / a0) / steps

    factor = 1 - 2 * G * 1.0 * 1.0 / 2.0 * math.sin(k) / k
    assert abs(decay_rate(G) / decay_rate(0.0) / factor - 1) < 3e-3


def test_poiseuille_profile_curvature(oracle_mod):
    """Plane Poiseuille flow between halfway walls: the steady velocity has
    constant second difference -g / (rho nu) with nu = (tau - 1/2)/3, and is
    symmetric about the channel centre."""
    L, g, tau = 12, 1e-6, 0.9
    p = W.params(lx=L, ly=1, lz=1, wall=(1, 0, 0), G=0.0, tau_s=tau, init_pert=0.0,
                 rho_a0=1.0, rho_b0=0.0, fluid_force=(0.0, 0.0, g))
    o = oracle_mod.Oracle(p)
    o.step(4000)
    f = o.get_f()
    rho = f.sum((0, 1)).reshape(L)
    uz = (np.einsum("li...,i->...", f, C[:, 2]).reshape(L) + 0.5 * g) / rho
    nu = (tau - 0.5) / 3
    d2 = uz[2:] - 2 * uz[1:-1] + uz[:-2]
    assert np.allclose(d2, -g / nu, rtol=2e-4)
    assert np.allclose(uz, uz[::-1], rtol=1e-9)


@pytest.mark.parametrize("tau_s,tau_g,steps", [(0.875, 1.0, 3000), (1.3, 0.734375, 3000), (0.9, 1.0, 3000),
                                               (0.6, 23 / 6, 6000)])
def test_poiseuille_with_halfway_walls_matches_the_two_rate_closed_form(oracle_mod, tau_s, tau_g, steps):
    """Steady plane Poiseuille flow with bounce-back walls at x = -1/2 and
    L - 1/2, in a scheme whose even non-conserved modes relax at tau_s and odd
    ones at tau_g (the MRT of Section 2 with a single component). The
    two-relaxation-time analysis of bounce-back (Ginzburg and d'Humieres 2003)
    gives the exact discrete profile
        u(x) = g / (2 nu) [(x + 1/2)(L - 1/2 - x) + (16 Lambda - 3) / 12],
    Lambda = (tau_s - 1/2)(tau_g - 1/2): the parabola of the halfway walls,
    with no slip at Lambda = 3/16 and a uniform slip otherwise. A wall at
    another place, a wrong rate on an odd mode or a wrong force term breaks it."""
    L, g = 8, 1e-6
    p = W.params(lx=L, ly=1, lz=1, wall=(1, 0, 0), G=0.0, tau_s=tau_s, tau_g=tau_g, init_pert=0.0,
                 rho_a0=1.0, rho_b0=0.0, fluid_force=(0.0, 0.0, g))
    o = oracle_mod.Oracle(p)
    o.step(steps)
    f = o.get_f()
    rho = f.sum((0, 1)).reshape(L)
    uz = (np.einsum("li...,i->...", f, C[:, 2]).reshape(L) + 0.5 * g) / rho
    nu = (tau_s - 0.5) / 3
    lam = (tau_s - 0.5) * (tau_g - 0.5)
    x = np.arange(L)
    want = g / (2 * nu) * ((x + 0.5) * (L - 0.5 - x) + (16 * lam - 3) / 12)
    assert np.allclose(uz, want, rtol=1e-9, atol=0)


# ---------------------------------------------------------------------------
# Fluctuation-dissipation (Section 2): noise only on non-conserved modes with
# variance 3 kT rho_l b_k; equipartition <j^2>/rho = kT per direction.
# ---------------------------------------------------------------------------
def test_mode_temperatures_of_a_thermalised_ideal_mixture_equal_kT(oracle_mod):
    """Fluctuation-dissipation (Section 2): in a thermalised ideal mixture
    (G = 0) the populations are independent Gaussians of variance
    3 kT rho_l w_i, so every non-conserved mode of either component holds
    <(m_k - m_k^eq)^2> = 3 kT rho_l b_k. The interdiffusion current holds
    kT rho_A rho_B / rho_tot and the total momentum kT rho_tot per axis.
    Halfway bounce-back only swaps populations of equal weight, so this holds
    next to walls too. The channel here is 4 x 5 nodes in cross-section
    between walls, so every node touches a wall. The oracle's temperature
    reductions must give kT within their statistical error (400 snapshots of
    800 nodes, sigma about 0.25 %; momentum relaxes slowly, so its
    snapshots are correlated and its tolerance is wider). A wrong mode norm
    or a missing factor fails this."""
    kT = 1e-4
    p = W.params(lx=4, ly=5, lz=40, wall=(1, 1, 0), G=0.0, kT=kT, init_pert=0.0)
    o = oracle_mod.Oracle(p)
    o.step(50)
    acc = []
    for _ in range(400):
        o.step(2)
        acc.append(o.mode_temps())
    mt = np.mean([a["mode_temp"] for a in acc], axis=0) / kT
    assert np.all(mt[:, :4] == 0.0)
    assert np.max(np.abs(mt[:, 4:] - 1.0)) < 0.015, mt
    dt = np.mean([a["diff_temp"] for a in acc], axis=0) / kT
    assert np.max(np.abs(dt - 1.0)) < 0.02, dt
    jt = np.mean([a["mom_temp"] for a in acc], axis=0) / kT
    assert np.max(np.abs(jt - 1.0)) < 0.03, jt
    assert acc[0]["n_bulk"] == 4 * 5 * 40


def test_mode_temperatures_of_a_uniform_flow_are_zero(oracle_mod):
    """A uniform equilibrium flow has no fluctuation: its modes equal the
    equilibrium ones and the two components move together. So every mode
    temperature and the interdiffusion temperature vanish, and the momentum
    temperature is the flow's rho_tot U_a^2. A sphere at rest in the flow
    removes its own nodes and their neighbours from the bulk count."""
    U = np.array([0.04, -0.03, 0.05])
    p = W.params(lx=12, ly=11, lz=13, wall=(0, 0, 0), G=0.0, init_pert=0.0, radius=2.6, pos0=(5.3, 5.1, 6.2))
    o = oracle_mod.Oracle(p)
    f = o.get_f()
    rho = (p["rho_a0"], p["rho_b0"])
    for l in range(2):
        f[l] = _feq(rho[l], U)[:, None, None, None] * np.ones((1, 13, 11, 12))
    o.set_f(f)
    t = o.mode_temps()
    assert np.max(np.abs(t["mode_temp"])) < 1e-28
    assert np.max(np.abs(t["diff_temp"])) < 1e-28
    assert np.allclose(t["mom_temp"], sum(rho) * U ** 2, rtol=1e-13, atol=0)
    solid = o.fields()["solid"]
    near = solid.copy()
    for c in C[1:].astype(int):
        near |= np.roll(solid, shift=(c[2], c[1], c[0]), axis=(0, 1, 2))
    assert t["n_bulk"] == int((~near).sum())


def test_single_node_mode_variances(oracle_mod):
    kT = 1e-4
    p = W.params(lx=1, ly=1, lz=1, wall=(0, 0, 0), G=0.0, kT=kT, init_pert=0.0, rho_a0=1.0, rho_b0=0.5)
    o = oracle_mod.Oracle(p)
    L = oracle_mod.lattice()
    e, b = L["e"], L["b"]
    n = 6000
    modes = np.empty((n, 2, 19))
    for s in range(n):
        o.step(1)
        f = o.get_f()[:, :, 0, 0, 0]
        modes[s] = f @ e.T
    rho = np.array([1.0, 0.5])
    # conserved: densities exactly, total momentum exactly
    assert np.allclose(modes[:, :, 0], rho, rtol=1e-12)
    assert np.abs(modes[:, 0, 1:4] + modes[:, 1, 1:4]).max() < 1e-14
    for l in range(2):
        var = (modes[:, l, 4:] ** 2).mean(0)
        want = 3 * kT * rho[l] * b[4:]
        assert np.all(np.abs(var / want - 1) < 5 * math.sqrt(2 / n))
    jvar = (modes[:, 0, 1:4] ** 2).mean(0)
    want = kT * rho[0] * rho[1] / rho.sum()
    assert np.all(np.abs(jvar / want - 1) < 5 * math.sqrt(2 / n))
    flat = modes[:, :, 4:].reshape(n, -1)
    corr = np.corrcoef(flat.T) - np.eye(flat.shape[1])
    assert np.abs(corr).max() < 6 / math.sqrt(n)


def test_single_node_relaxation_rates_and_stationary_variances(oracle_mod):
    """With separate relaxation times for the stress, the component-momentum
    and the ghost modes (the MRT of Section 2), one node of a 1x1x1 periodic
    box (streaming maps it onto itself) makes every non-conserved mode a
    discrete Ornstein-Uhlenbeck process m' = gamma_k m + noise with
    gamma_k = 1 - 1/tau_k. Its lag-one autocorrelation is gamma_k, which pins
    which modes relax at which rate. Its stationary variance is still
    3 kT rho_l b_k (the interdiffusion current's kT rho_A rho_B / rho), as
    fluctuation-dissipation requires whatever the rates."""
    kT, taus, n = 1e-4, {"tau_s": 0.8, "tau_d": 0.7, "tau_g": 1.3}, 8000
    p = W.params(lx=1, ly=1, lz=1, wall=(0, 0, 0), G=0.0, kT=kT, init_pert=0.0, rho_a0=1.0, rho_b0=0.5, **taus)
    o = oracle_mod.Oracle(p)
    L = oracle_mod.lattice()
    e, b = L["e"], L["b"]
    modes = np.empty((n, 2, 19))
    for s in range(n):
        o.step(1)
        modes[s] = o.get_f()[:, :, 0, 0, 0] @ e.T
    rho = np.array([1.0, 0.5])
    gamma = np.array([0.0] * 4 + [1 - 1 / taus["tau_s"]] * 6 + [1 - 1 / taus["tau_g"]] * 9)
    gamma[1:4] = 1 - 1 / taus["tau_d"]
    want_var = 3 * kT * np.outer(rho, b)
    want_var[:, 1:4] = kT * rho[0] * rho[1] / rho.sum()
    for l in range(2):
        for k in range(1, 19):
            m = modes[:, l, k]
            var = (m ** 2).mean()
            ac = (m[1:] * m[:-1]).mean() / var
            g = gamma[k]
            assert abs(ac - g) < 5 / math.sqrt(n), (l, k, ac, g)
            assert abs(var / want_var[l, k] - 1) < 5 * math.sqrt(2 * (1 + g * g) / (1 - g * g) / n), (l, k)


@pytest.mark.slow
def test_fluid_equipartition(oracle_mod):
    kT = 1e-4
    p = W.params(lx=6, ly=6, lz=6, wall=(0, 0, 0), G=0.0, kT=kT, init_pert=0.0, rho_a0=1.0, rho_b0=0.3)
    o = oracle_mod.Oracle(p)
    o.step(50)
    acc, cnt = np.zeros(3), 0
    for _ in range(150):
        o.step(1)
        f = o.get_f()
        rho = f.sum((0, 1))
        j = np.einsum("li...,ia->a...", f, C)
        acc += (j ** 2 / rho).mean((1, 2, 3))
        cnt += 1
    assert np.allclose(acc / cnt, kT, rtol=0.05)


def test_sphere_comoving_with_uniform_flow_is_invisible(oracle_mod):
    """Galilean invariance of the moving-wall link rule (Ladd 1994, cited in
    Section 2): in a uniform flow U with the sphere moving at U (no wetting
    shift), the bounced populations equal the equilibrium ones the solid would
    have sent, so the exchanged force and torque vanish and the flow is left
    unchanged. A wrong factor or sign in the moving-wall term fails this."""
    drho = 0.0
    U = np.array([0.013, -0.021, 0.017])
    p = W.params(lx=12, ly=11, lz=13, wall=(0, 0, 0), G=1.2, init_pert=0.0, radius=3.1,
                 delta_rho=drho, pos0=(5.37, 4.81, 6.22))
    o = oracle_mod.Oracle(p)
    f = o.get_f()
    for l, r in enumerate((p["rho_a0"], p["rho_b0"])):
        f[l] = _feq(r, U)[:, None, None, None] * np.ones((1, 13, 11, 12))
    o.set_f(f)
    o.set_particle(p["pos0"], V=U)
    solid0 = o.fields()["solid"].copy()
    o.step(1)
    pa = o.particle()
    assert np.abs(pa["F"]).max() < 1e-14
    assert np.abs(pa["T"]).max() < 1e-13
    g = o.get_f()
    keep = ~(solid0 | o.fields()["solid"])
    for l in range(2):
        assert np.allclose(g[l][:, keep], f[l][:, keep], rtol=0, atol=1e-15)


@pytest.mark.parametrize("G", [0.0, 1.2])
def test_uncovered_nodes_are_refilled_with_the_comoving_flow(oracle_mod, G):
    """Cover and uncover (Section 2, particle paragraph) leave a flow that
    moves with the sphere unchanged. The fluid starts each step exactly
    uniform at f_eq(rho_l, U) and the sphere moves at U. The particle nodes
    hold arbitrary values, since their populations are not part of the state.
    After one step every fluid node, newly uncovered ones included, must hold
    f_eq(rho_l, U) again.

    So the refill of an uncovered node must use the sphere's surface velocity
    and the density of its fluid neighbours. A refill at rest fails this. So
    does a mean that takes in particle nodes or other uncovered nodes (they
    hold the arbitrary values). The step's ledgers must also match exactly:
    the mass ledger is rho_l (covered - uncovered), the pending impulse is
    rho_tot U (covered - uncovered), and force and torque vanish. The
    sphere is stepped along a trajectory X_k = X_0 + k U, one fresh step per
    position, so that each step meets different cover and uncover sets.
    Only the translational part of the surface velocity is pinned here (the
    sphere does not spin)."""
    U = np.array([0.29, -0.23, 0.31])
    L = (16, 15, 17)
    X0 = np.array([7.13, 6.71, 8.37])
    rho = (1.0, 0.05)
    rng = np.random.default_rng(5)
    n_cov = n_unc = 0
    for k in range(8):
        X = np.mod(X0 + k * U, L)
        p = W.params(lx=L[0], ly=L[1], lz=L[2], wall=(0, 0, 0), G=G, init_pert=0.0, radius=3.3,
                     rho_p_ratio=2.0, delta_rho=0.0, pos0=tuple(X))
        o = oracle_mod.Oracle(p)
        o.set_particle(X, V=U)
        solid0 = o.fields()["solid"].copy()
        f = np.empty((2, 19, L[2], L[1], L[0]))
        for l in range(2):
            f[l] = _feq(rho[l], U)[:, None, None, None]
            f[l][:, solid0] = rng.uniform(0.0, 3.0, size=(19, int(solid0.sum())))
        o.set_f(f)
        o.step(1)
        pa = o.particle()
        assert np.allclose(pa["V"], U, rtol=0, atol=1e-16)
        assert np.abs(pa["F"]).max() < 1e-13
        assert np.abs(pa["T"]).max() < 1e-12
        solid1 = o.fields()["solid"]
        cov = int((solid1 & ~solid0).sum())
        unc = int((solid0 & ~solid1).sum())
        n_cov += cov
        n_unc += unc
        g = o.get_f()
        fluid = ~solid1
        for l in range(2):
            assert np.allclose(g[l][:, fluid], _feq(rho[l], U)[:, None], rtol=0, atol=2e-15), (k, l)
            assert abs(pa["delta"][l] * pa["nfluid"] - rho[l] * (cov - unc)) < 1e-13
        assert np.allclose(pa["Ppend"], sum(rho) * U * (cov - unc), rtol=0, atol=1e-13)
    assert n_unc >= 40 and n_cov >= 40, (n_cov, n_unc)


# ---------------------------------------------------------------------------
# Brute force on a 4^3 box
# ---------------------------------------------------------------------------
def test_full_step_on_a_4cubed_box_equals_population_space_bgk(oracle_mod):
    """Three noise-free steps of a periodic 4x4x4 two-component box with the
    Shan-Chen force, against a brute-force numpy step written in population
    space: with every relaxation time 1 the MRT collision is BGK with tau = 1,
    f* = f_eq(rho_l, u) + S_l / 2 with Guo's source
    S_li = w_i [3 (c_i - u) . F_l + 9 (c_i . u)(c_i . F_l)], u = v^(H), and
    streaming is a periodic shift of each direction by c_i."""
    p = W.params(lx=4, ly=4, lz=4, wall=(0, 0, 0), G=1.2, kT=0.0)
    f = W.random_populations(p, 44, amp=0.1, vel=0.05)
    o = oracle_mod.Oracle(p)
    o.set_f(f)
    o.step(3)
    w = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
    G = p["G"]

    def shifted(a, c):  # a(x + c) on the periodic box, arrays indexed [z, y, x]
        return np.roll(a, shift=(-int(c[2]), -int(c[1]), -int(c[0])), axis=(0, 1, 2))

    for _ in range(3):
        rho = f.sum(axis=1)                                    # (2, z, y, x)
        j = np.einsum("lizyx,ia->lazyx", f, C)                 # (2, 3, z, y, x)
        gsum = np.zeros_like(j)                                # sum_i w_i psi_other(x + c_i) c_i
        for i in range(1, 19):
            for l in range(2):
                gsum[l] += w[i] * shifted(rho[1 - l], C[i])[None] * C[i][:, None, None, None]
        F = -G * rho[:, None] * gsum
        u = (j.sum(axis=0) + 0.5 * F.sum(axis=0)) / rho.sum(axis=0)
        cu = np.einsum("ia,azyx->izyx", C, u)
        uu = (u * u).sum(axis=0)
        new = np.empty_like(f)
        for l in range(2):
            feq = w[:, None, None, None] * rho[l][None] * (1 + 3 * cu + 4.5 * cu ** 2 - 1.5 * uu[None])
            cF = np.einsum("ia,azyx->izyx", C, F[l])
            uF = (u * F[l]).sum(axis=0)
            S = w[:, None, None, None] * (3 * (cF - uF[None]) + 9 * cu * cF)
            fs = feq + 0.5 * S
            for i in range(19):
                new[l, i] = shifted(fs[i], -C[i])  # f(x + c_i) <- f*(x)
        f = new
    assert np.allclose(o.get_f(), f, rtol=1e-13, atol=1e-16)


# ---------------------------------------------------------------------------
# Particle hydrodynamics and fluctuations
# ---------------------------------------------------------------------------
def _hasimoto_K(R, L):
    """Drag factor of a simple cubic array of spheres (Hasimoto 1959):
    F = 6 pi eta R U K, 1/K = 1 - 1.7601 c^(1/3) + c - 1.5593 c^2, c the
    volume fraction."""
    c = 4 / 3 * math.pi * R ** 3 / L ** 3
    return 1 / (1 - 1.7601 * c ** (1 / 3) + c - 1.5593 * c ** 2)


def test_settling_drag_of_a_sphere_in_a_periodic_box(oracle_mod):
    """Noise-free sphere (R = 2.5) driven through a periodic 16^3 box, with the
    counterforce on the fluid so that the system reaches a steady state.
    The steady velocity relative to the fluid, read through Stokes' law with
    Hasimoto's periodic-array correction and eta = rho nu = rho_tot / 6 (tau = 1),
    gives the sphere's hydrodynamic radius: it must lie within half a lattice
    spacing below and a full spacing above the nominal radius (bounce-back
    spheres are known to act slightly smaller or larger than R)."""
    R, L = 2.5, 16
    p = W.params(lx=L, ly=L, lz=L, wall=(0, 0, 0), radius=R, rho_p_ratio=1.5, g=4e-4, kT=0.0, init_pert=0.0,
                 G=0.0, fluid_counterforce=1)
    o = oracle_mod.Oracle(p)
    o.step(600)
    us, uf = [], []
    for _ in range(40):
        o.step(10)
        pa, ob = o.particle(), o.observables()
        us.append(pa["V"][2])
        uf.append(ob["momentum"][2] / ob["mass"].sum())
    U = float(np.mean(us) - np.mean(uf))
    eta = (p["rho_a0"] + p["rho_b0"]) / 6
    F = o.particle()["Fp"]
    Rh = R
    for _ in range(60):
        Rh = F / (6 * math.pi * eta * U * _hasimoto_K(Rh, L))
    assert U > 0
    assert R - 0.5 <= Rh <= R + 1.0, f"hydrodynamic radius {Rh:.3f} for R = {R}"
    assert np.std(us) < 0.05 * abs(np.mean(us))  # steady


def test_particle_velocity_equipartition(oracle_mod):
    """A heavy sphere (rho_p = 5 rho, R = 2.5) in a fluctuating 12^3 channel
    without driving: its velocity variance per axis is kT / m_p (the paper's
    Langevin picture, Section 3). For light spheres the explicit time stepping
    of the coupling biases the leap-frog velocities (about +30 % for the
    half-step velocity, -10 % for the step average at rho_p = 1.5 rho); with a
    long particle relaxation time both estimates must be within 15 %."""
    p = W.params(lx=12, ly=12, lz=12, wall=(1, 1, 0), radius=2.5, rho_p_ratio=5.0, g=0.0, kT=1e-4, init_pert=0.0,
                 G=0.0)
    o = oracle_mod.Oracle(p)
    o.step(300)
    v, va = [], []
    for _ in range(3000):
        o.step(1)
        pa = o.particle()
        v.append(pa["V"].copy())
        va.append(pa["Vavg"].copy())
    s = p["kT"] / o.particle()["mp"]
    rv = float(np.mean(np.var(v, axis=0)) / s)
    ra = float(np.mean(np.var(va, axis=0)) / s)
    assert 0.85 <= rv <= 1.15, rv
    assert 0.85 <= ra <= 1.15, ra


@pytest.mark.parametrize("drho", [0.2, -0.2])
def test_wetting_shift_enriches_the_preferred_component_at_the_surface(oracle_mod, drho):
    """The sign convention of the wetting parameter (Section 2: the virtual
    layer carries the neighbour mean plus delta_rho for A, minus for B).
    delta_rho > 0 makes the particle hydrophilic to A: after relaxation the
    fluid nodes touching a fixed sphere hold more A and less B than the fluid
    far from it; delta_rho < 0 the reverse. Total mass stays exact."""
    p = W.params(lx=14, ly=14, lz=14, wall=(0, 0, 0), radius=2.5, rho_p_ratio=1e9, g=0.0, kT=0.0, init_pert=0.0,
                 rho_a0=0.6, rho_b0=0.4, G=1.2, delta_rho=drho, pos0=(6.5, 6.5, 6.5))
    o = oracle_mod.Oracle(p)
    m0 = o.observables()["mass"]
    o.step(300)
    fl = o.fields()
    solid = fl["solid"]
    touch = np.zeros_like(solid)
    for c in C[1:]:
        touch |= np.roll(solid, shift=(int(c[2]), int(c[1]), int(c[0])), axis=(0, 1, 2))
    touch &= ~solid
    zz, yy, xx = np.meshgrid(np.arange(14), np.arange(14), np.arange(14), indexing="ij")
    r2 = (xx - 6.5) ** 2 + (yy - 6.5) ** 2 + (zz - 6.5) ** 2
    far = r2 > 6.0 ** 2
    ra, rb = fl["rho"][0], fl["rho"][1]
    sgn = np.sign(drho)
    assert sgn * (ra[touch].mean() - ra[far].mean()) > 1e-3, (ra[touch].mean(), ra[far].mean())
    assert sgn * (rb[touch].mean() - rb[far].mean()) < -1e-3, (rb[touch].mean(), rb[far].mean())
    assert np.allclose(o.observables()["mass"], m0, rtol=1e-12)


def test_static_structure_factor_is_flat(oracle_mod):
    """Fluctuation-dissipation at every wavelength (Section 2): in a
    fluctuating ideal mixture (G = 0) the equal-time spectra of the density
    and momentum fluctuations are flat, <|drho_k|^2>/N = 3 kT rho (per
    component and in total) and <|j_k|^2>/N = kT rho_tot per axis, because the
    noise thermalises every non-conserved mode, ghosts included. Checked on
    every wavevector of an 8^3 box off the Nyquist planes, shell by shell."""
    kT = 1e-4
    p = W.params(lx=8, ly=8, lz=8, wall=(0, 0, 0), G=0.0, kT=kT, init_pert=0.0, rho_a0=1.0, rho_b0=0.3)
    o = oracle_mod.Oracle(p)
    o.step(100)
    S = {"rho": np.zeros((8, 8, 8)), "rhoA": np.zeros((8, 8, 8)), "j": np.zeros((8, 8, 8))}
    n = 1000
    for _ in range(n):
        o.step(1)
        f = o.get_f()
        rho, ra = f.sum((0, 1)), f[0].sum(0)
        j = np.einsum("li...,ia->a...", f, C)
        S["rho"] += np.abs(np.fft.fftn(rho - rho.mean())) ** 2 / rho.size
        S["rhoA"] += np.abs(np.fft.fftn(ra - ra.mean())) ** 2 / rho.size
        S["j"] += sum(np.abs(np.fft.fftn(j[a])) ** 2 for a in range(3)) / (3 * rho.size)
    want = {"rho": 3 * kT * 1.3, "rhoA": 3 * kT * 1.0, "j": kT * 1.3}
    kz, ky, kx = np.meshgrid(np.arange(8), np.arange(8), np.arange(8), indexing="ij")
    fold = [np.minimum(k, 8 - k) for k in (kx, ky, kz)]
    k2 = sum(k * k for k in fold)
    keep = (k2 > 0) & np.all([k != 4 for k in fold], axis=0)
    for name, s in S.items():
        r = s / n / want[name]
        shells = [r[keep & (k2 == q)].mean() for q in np.unique(k2[keep])]
        assert abs(r[keep].mean() - 1.0) < 0.03, (name, r[keep].mean())
        assert all(abs(v - 1.0) < 0.15 for v in shells), (name, np.round(shells, 3))  # about 4 sigma at k^2 = 1


def test_sphere_corotating_with_rigidly_rotating_fluid_feels_no_torque(oracle_mod):
    """The moving link rule (Section 2) with rotation: fluid in rigid rotation
    Omega about the sphere's centre (equilibrium populations at u = Omega x r)
    exerts no torque on a sphere spinning with the same Omega; on a sphere at
    rest it exerts a torque along Omega. After one step the co-rotating torque
    and force are below 1e-3 of the resting sphere's torque (a wrong lever,
    surface velocity or sign in the link rule gives a ratio of order one)."""
    L = 16
    X = np.array([7.3, 7.6, 7.45])
    Om = np.array([0.0005, -0.0003, 0.002])
    p = W.params(lx=L, ly=L, lz=L, wall=(0, 0, 0), G=0.0, kT=0.0, init_pert=0.0, radius=3.3, pos0=tuple(X))
    w = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
    zz, yy, xx = np.meshgrid(np.arange(L), np.arange(L), np.arange(L), indexing="ij")
    r = np.stack([xx - X[0], yy - X[1], zz - X[2]], 0)
    u = np.cross(Om[:, None, None, None], r, axis=0)
    cu = np.einsum("ia,a...->i...", C.astype(float), u)
    feq = w[:, None, None, None] * (1 + 3 * cu + 4.5 * cu ** 2 - 1.5 * (u ** 2).sum(0))
    f = np.stack([p["rho_a0"] * feq, p["rho_b0"] * feq], 0)

    def after_one_step(om_p):
        o = oracle_mod.Oracle(p)
        o.set_f(f)
        o.set_particle(tuple(X), (0.0, 0.0, 0.0), tuple(om_p))
        o.step(1)
        return o.particle()

    co, rest = after_one_step(Om), after_one_step((0.0, 0.0, 0.0))
    Tref = np.linalg.norm(rest["T"])
    assert np.dot(rest["T"], Om) > 0.9 * Tref * np.linalg.norm(Om)  # dragged along the rotation
    assert np.linalg.norm(co["T"]) < 1e-3 * Tref
    assert np.linalg.norm(co["F"]) < 1e-3 * Tref


@pytest.mark.parametrize("G,drho", [(0.0, 0.0), (1.2, 0.3), (1.2, -0.3)])
def test_angular_momentum_about_the_sphere_is_conserved(oracle_mod, G, drho):
    """Every exchange in the step is central or local: collision keeps each
    node's momentum, streaming moves a population along its own velocity, the
    link rule hands the particle (f_out + f_back) c_i across a link whose
    midpoint and fluid end differ by a multiple of c_i, and the Shan-Chen
    pair forces, including the reaction of the virtual layer on the particle
    (Section 2), act along the link that joins the pair. So the fluid's
    angular momentum about the sphere's centre changes by minus the torque the
    sphere receives, exactly, as long as the disturbance has not reached the
    periodic boundary. A sphere spinning in fluid at rest, heavy enough not to
    move, checks that over three steps."""
    L, R, X = 24, 3.3, np.array([11.6, 12.2, 11.9])
    p = W.params(lx=L, ly=L, lz=L, wall=(0, 0, 0), G=G, delta_rho=drho, init_pert=0.0, radius=R,
                 rho_p_ratio=1e12, g=0.0, kT=0.0)
    o = oracle_mod.Oracle(p)
    o.set_particle(X, V=(0.0, 0.0, 0.0), Omega=(0.003, -0.002, 0.004))
    z, y, x = np.indices((L, L, L))
    arm = np.stack([x, y, z], axis=-1) - X
    arm -= L * np.round(arm / L)

    def fluid_angular_momentum():
        j = np.einsum("li...,ia->...a", o.get_f(), C)
        j[o.fields()["solid"].astype(bool)] = 0.0
        return np.cross(arm, j).sum(axis=(0, 1, 2))

    L0 = fluid_angular_momentum()
    torque = np.zeros(3)
    for _ in range(3):
        o.step(1)
        torque += o.particle()["T"]
    assert np.linalg.norm(torque) > 1.0
    assert np.abs(fluid_angular_momentum() - L0 + torque).max() < 1e-12 * np.linalg.norm(torque)


def _direction_map(M):
    """Index of M c_i in the lattice, for each direction i."""
    Ci = C.astype(int)
    return np.array([int(np.flatnonzero((Ci == M @ Ci[i]).all(axis=1))[0]) for i in range(19)])


def test_square_channel_symmetry_is_kept_through_cover_and_uncover(oracle_mod):
    """The step commutes with the symmetries of the square channel (walls on
    x and y) about its axis: the mirrors x -> L-1-x and y -> L-1-y and the swap
    x <-> y, each acting on positions and on the velocity set. A state with
    that symmetry, a wetted sphere (G = 1.2, Delta rho = 0.3) on the axis
    moving along it, keeps it exactly, through the Shan-Chen force, the wall
    ghosts, the virtual layer, the link rule and the cover/uncover events of a
    settling sphere; and the sphere stays on the axis without spin. A
    direction or an axis handled unlike its images breaks it."""
    L, Lz = 10, 16
    p = W.params(lx=L, ly=L, lz=Lz, wall=(1, 1, 0), G=1.2, delta_rho=0.3, radius=2.6, rho_p_ratio=1.5, g=2e-3,
                 kT=0.0, init_pert=0.0)
    mx = _direction_map(np.diag([-1, 1, 1]))
    my = _direction_map(np.diag([1, -1, 1]))
    sw = _direction_map(np.array([[0, 1, 0], [1, 0, 0], [0, 0, 1]]))

    def mirror_x(f):
        g = np.empty_like(f)
        g[:, mx] = f[..., ::-1]
        return g

    def mirror_y(f):
        g = np.empty_like(f)
        g[:, my] = f[..., ::-1, :]
        return g

    def swap_xy(f):
        g = np.empty_like(f)
        g[:, sw] = np.swapaxes(f, -1, -2)
        return g

    f = W.random_populations(p, 11)
    images = [f, swap_xy(f)]
    images += [mirror_x(g) for g in images]
    images += [mirror_y(g) for g in images]
    f = sum(images) / len(images)  # average over the eight symmetries of the square
    o = oracle_mod.Oracle(p)
    o.set_f(f)
    o.set_particle(((L - 1) / 2, (L - 1) / 2, 7.3), V=(0.0, 0.0, 0.05))
    nfluid = set()
    for _ in range(60):
        o.step(1)
        nfluid.add(o.particle()["nfluid"])
    assert len(nfluid) > 1  # nodes were covered and uncovered
    g = o.get_f()
    for T in (mirror_x, mirror_y, swap_xy):
        assert np.abs(T(g) - g).max() < 1e-13 * np.abs(g).max()
    pa = o.particle()
    assert np.abs(pa["X"][:2] - (L - 1) / 2).max() < 1e-13
    assert np.abs(pa["V"][:2]).max() < 1e-15 and np.abs(pa["Omega"]).max() < 1e-15


def test_component_exchange_with_a_mirror_is_kept_at_an_interface(oracle_mod):
    """The two components enter the method symmetrically (Section 2: one G,
    psi = rho, the same relaxation times; Delta rho = 0 wets neither). So
    exchanging A and B together with the mirror through a flat A/B interface
    (z -> 7 - z, c_z -> -c_z, A-rich layer onto B-rich layer) is a symmetry
    of the step. A separated mixture (G = 1.5, the printed 2.21/0.09,
    perturbed, then symmetrised) with a sphere on the interface, in a square
    channel with distinct stress, interdiffusion and ghost rates, moving along
    the interface through cover and uncover events, keeps it exactly: the
    sphere stays on the interface and spins only about its normal. A
    component treated unlike the other breaks it."""
    L, Lz = 10, 16
    p = W.params(lx=L, ly=L, lz=Lz, wall=(1, 1, 0), G=1.5, delta_rho=0.0, radius=2.7, rho_p_ratio=1.5, g=0.0,
                 kT=0.0, init_pert=0.0, rho_a0=2.21, rho_b0=0.09, tau_s=0.8, tau_d=0.7, tau_g=1.3)
    mz = _direction_map(np.diag([1, 1, -1]))
    zmap = (7 - np.arange(Lz)) % Lz

    def exchange(f):
        g = np.empty_like(f)
        g[:, mz] = f[:, :, zmap]
        return g[::-1]

    f = W.layered_populations(p, lo=4, hi=12)
    f = f * (1 + 0.01 * np.random.default_rng(3).standard_normal(f.shape))
    f = 0.5 * (f + exchange(f))
    o = oracle_mod.Oracle(p)
    o.set_f(f)
    o.set_particle(((L - 1) / 2, (L - 1) / 2, 3.5), V=(0.12, -0.06, 0.0), Omega=(0.0, 0.0, 0.003))
    nfluid = set()
    for _ in range(60):
        o.step(1)
        nfluid.add(o.particle()["nfluid"])
    assert len(nfluid) > 1  # nodes were covered and uncovered
    g = o.get_f()
    assert np.abs(exchange(g) - g).max() < 1e-13 * np.abs(g).max()
    pa = o.particle()
    assert abs(pa["X"][2] - 3.5) < 1e-13 and abs(pa["V"][2]) < 1e-15
    assert np.abs(pa["Omega"][:2]).max() < 1e-15
