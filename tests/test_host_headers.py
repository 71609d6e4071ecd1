"""Header functions of the step kernels, checked on the host (no GPU).

The programs include the library's headers and run the helpers the
kernels call, on random lattices, wall flags, radii and positions, against a
brute-force scan of the lattice:

* tests/host_tiles.cu (box_origin, box_node_inside, tile_near, adj_edge_candidate, adj_edge_node,
  candidate_tile, make_kparams, both tile policies): the particle box holds
  exactly the sphere's nodes, every fluid node next to the sphere is in a
  near tile, and the near launch reaches every near tile exactly once;
* tests/host_shell.cu (shell_node, virtual_node): every shell node of the
  padded density field holds its periodic image or its wall-ghost mean, every
  particle node with fluid neighbours holds the virtual-layer value, in
  either order of the two, and the padding columns are never written;
* tests/host_philox.cu (philox4x32_10, philox_rk with the round keys that
  make_kparams precomputes, uniform_open): the published Philox4x32-10
  known-answer vectors, agreement of the two Philox forms on random keys and
  counters, and the exact uniform map;
* tests/host_modes.cu (to_modes, from_modes, bnorm): the collision's
  hand-factored transforms against the D3Q19 mode basis written out from its
  polynomials, exactly, and their round trip;
* tests/host_fused.cu (DensitySink, gather_column, roll_update, put_density,
  FinishItems, finish_node, near_dilated, near_box_axis): the fused collide's
  data flow replayed block by block on random lattices, planes per block and
  particle boxes gives every node outside the near-particle region the direct
  sum of the 19 values pushed into it, each such node completed once, and the
  near-particle region lies in the box its recompute walks;
* tests/host_push.cu (PushFrame::target): the push target of every
  population of every node equals the target taken from the definition
  (x + c_i with wrap, or the node itself in the opposite direction across a
  wall);
* tests/host_groups.cu (group_by_blocks): the ensemble's descriptor-chunk
  bulk launches take every replica exactly once, at most the cap per
  launch, with a grid that covers every member's tiles and at most a quarter
  of its blocks idle, and start a new launch only when they must;
* tests/host_restore.cu (check_restored_state): a particle record read from
  a checkpoint passes when it is one the library wrote, and is refused when
  its mask index, centre, velocities, box origin, fluid count, step or mass
  correction is corrupt, before any of it reaches the device.
"""
import os
import subprocess

from paper_1909_01092_gb300 import build

HERE = os.path.dirname(os.path.abspath(__file__))


def _build_and_run(tmp_path, name, arg):
    exe = str(tmp_path / name)
    cmd = [build.nvcc(), *build.ARCH_FLAGS, "-O2", "-std=c++17", "-I", build.INCLUDE, "-I", build.CSRC,
           "-o", exe, os.path.join(HERE, name + ".cu")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    r = subprocess.run([exe, str(arg)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    return r.stdout


def test_near_tiles_cover_the_sphere_exactly_once(tmp_path):
    out = _build_and_run(tmp_path, "host_tiles", 600)
    assert "configurations 1200 failed 0" in out, out


def test_shell_and_virtual_layer_of_the_padded_density_field(tmp_path):
    out = _build_and_run(tmp_path, "host_shell", 300)
    words = out.split()
    run, failed, with_particle = (int(words[words.index(w) + 1]) for w in ("configurations", "failed", "with_particle"))
    assert failed == 0 and run > 300 and with_particle > run // 2, out


def test_cuda_philox_matches_the_published_known_answers(tmp_path):
    out = _build_and_run(tmp_path, "host_philox", os.path.join(HERE, "golden", "philox4x32_10_kat.txt"))
    assert "kat_rows 3 draws 80000 failed 0" in out, out


def test_collision_mode_transforms_match_the_basis_polynomials(tmp_path):
    out = _build_and_run(tmp_path, "host_modes", "")
    assert "failed 0" in out, out


def test_restored_particle_records_are_checked(tmp_path):
    out = _build_and_run(tmp_path, "host_restore", "")
    words = out.split()
    configs, refused, failed = (int(words[words.index(w) + 1]) for w in ("configurations", "refused", "failed"))
    assert failed == 0 and configs > 300 and refused > 6 * configs, out


def test_fused_density_bookkeeping_gives_the_direct_sums(tmp_path):
    out = _build_and_run(tmp_path, "host_fused", 300)
    words = out.split()
    run, failed, with_particle = (int(words[words.index(w) + 1]) for w in ("configurations", "failed", "with_particle"))
    assert failed == 0 and run == 300 and with_particle > 100, out


def test_push_targets_follow_streaming_and_bounce_back(tmp_path):
    out = _build_and_run(tmp_path, "host_push", "")
    words = out.split()
    configs, targets, failed = (int(words[words.index(w) + 1]) for w in ("configurations", "targets", "failed"))
    assert failed == 0 and configs > 250 and targets > 10 ** 6, out


def test_ensemble_launch_groups(tmp_path):
    out = _build_and_run(tmp_path, "host_groups", 2000)
    assert "cases 2000 failed 0" in out, out
