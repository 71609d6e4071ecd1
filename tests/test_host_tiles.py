"""Tile classification of the step kernels, checked on the host (no GPU).

tests/host_tiles.cu includes the library's headers and runs the geometry
helpers the kernels call (box_origin, box_node_inside, tile_near,
candidate_tile, make_kparams) on random lattices, walls, radii, positions and
tile policies, against a brute-force scan of the lattice: the particle box
holds exactly the sphere's nodes, every fluid node next to the sphere is in a
near tile, and the near launch reaches every near tile exactly once.
"""
import os
import subprocess

from paper_1909_01092_gb300 import build

HERE = os.path.dirname(os.path.abspath(__file__))


def test_near_tiles_cover_the_sphere_exactly_once(tmp_path):
    exe = str(tmp_path / "host_tiles")
    cmd = [build.nvcc(), *build.ARCH_FLAGS, "-O2", "-std=c++17", "-I", build.INCLUDE, "-I", build.CSRC,
           "-o", exe, os.path.join(HERE, "host_tiles.cu")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    r = subprocess.run([exe, "600"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "failed 0" in r.stdout and "configurations 1200" in r.stdout, r.stdout
