"""Host check of the node-level collision adjoint the CUDA adjoint kernels use
(paper_1909_01092_gb300/csrc/flbm_adjoint_math.h): adj_modes must be the
transpose of the Jacobian of fwd_modes. Compiled here with g++ in double
precision; checked against central finite differences of fwd_modes through
the identity <lambda, J v> = <J^T lambda, v> for random lambda and v.

Also the double-float arithmetic (csrc/flbm_df.h) the adjoint uses for its
large parts: each operation against exact rational arithmetic, and
adj_modes_ab evaluated in it against the double evaluation."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1909_01092_gb300", "csrc")

SHIM = r"""
#include "flbm_adjoint_math.h"
#include "flbm_df.h"
extern "C" void df_op(int op, const float* a, const float* b, float* out) {
    const flbm::df x(a[0], a[1]), y(b[0], b[1]);
    const flbm::df r = op == 0 ? x + y : op == 1 ? x - y : op == 2 ? x * y : op == 3 ? x / y
                     : op == 4 ? x + b[0] : x * b[0];
    out[0] = r.hi; out[1] = r.lo;
}
extern "C" void adj_ab_df(const double* in, double G, const double* ab, double* out) {
    using flbm::df;
    const df rho[2] = {df(in[0]), df(in[1])};
    const df j[2][3] = {{df(in[2]), df(in[3]), df(in[4])}, {df(in[5]), df(in[6]), df(in[7])}};
    const df g[2][3] = {{df(in[8]), df(in[9]), df(in[10])}, {df(in[11]), df(in[12]), df(in[13])}};
    const df ext[3] = {df(in[14]), df(in[15]), df(in[16])};
    const df a[2] = {df(ab[0]), df(ab[1])};
    const df b[2][3] = {{df(ab[2]), df(ab[3]), df(ab[4])}, {df(ab[5]), df(ab[6]), df(ab[7])}};
    df lrho[2], lj[2][3], lg[2][3], lG;
    flbm::adj_modes_ab<df>(rho, j, g, ext, df(G), a, b, lrho, lj, lg, lG);
    out[0] = lrho[0].value(); out[1] = lrho[1].value();
    for (int l = 0; l < 2; ++l) for (int c = 0; c < 3; ++c) { out[2 + 3 * l + c] = lj[l][c].value(); out[8 + 3 * l + c] = lg[l][c].value(); }
    out[14] = lG.value();
}
extern "C" void adj_ab_mixed(const float* in, float G, const double* ab, int use_df, double* out) {
    using flbm::df;
    const float rho[2] = {in[0], in[1]};
    const float j[2][3] = {{in[2], in[3], in[4]}, {in[5], in[6], in[7]}};
    const float g[2][3] = {{in[8], in[9], in[10]}, {in[11], in[12], in[13]}};
    const float ext[3] = {in[14], in[15], in[16]};
    if (use_df) {
        const df a[2] = {df(ab[0]), df(ab[1])};
        const df b[2][3] = {{df(ab[2]), df(ab[3]), df(ab[4])}, {df(ab[5]), df(ab[6]), df(ab[7])}};
        df lrho[2], lj[2][3], lg[2][3], lG;
        flbm::adj_modes_ab_mixed<df>(rho, j, g, ext, G, a, b, lrho, lj, lg, lG);
        out[0] = lrho[0].value(); out[1] = lrho[1].value();
        for (int l = 0; l < 2; ++l) for (int c = 0; c < 3; ++c) { out[2 + 3 * l + c] = lj[l][c].value(); out[8 + 3 * l + c] = lg[l][c].value(); }
        out[14] = lG.value();
    } else {
        const double a[2] = {(double)df(ab[0]).value(), (double)df(ab[1]).value()};
        double b[2][3];
        for (int l = 0; l < 2; ++l) for (int c = 0; c < 3; ++c) b[l][c] = df(ab[2 + 3 * l + c]).value();
        double lrho[2], lj[2][3], lg[2][3], lG;
        flbm::adj_modes_ab_mixed<double>(rho, j, g, ext, G, a, b, lrho, lj, lg, lG);
        out[0] = lrho[0]; out[1] = lrho[1];
        for (int l = 0; l < 2; ++l) for (int c = 0; c < 3; ++c) { out[2 + 3 * l + c] = lj[l][c]; out[8 + 3 * l + c] = lg[l][c]; }
        out[14] = lG;
    }
}
extern "C" void fwd(const double* in, double G, double* ms) {
    const double rho[2] = {in[0], in[1]};
    const double j[2][3] = {{in[2], in[3], in[4]}, {in[5], in[6], in[7]}};
    const double g[2][3] = {{in[8], in[9], in[10]}, {in[11], in[12], in[13]}};
    const double ext[3] = {in[14], in[15], in[16]};
    double m[2][10];
    flbm::fwd_modes<double>(rho, j, g, ext, G, m);
    for (int l = 0; l < 2; ++l) for (int k = 0; k < 10; ++k) ms[10 * l + k] = m[l][k];
}
extern "C" void adj(const double* in, double G, const double* lmf, double* out) {
    const double rho[2] = {in[0], in[1]};
    const double j[2][3] = {{in[2], in[3], in[4]}, {in[5], in[6], in[7]}};
    const double g[2][3] = {{in[8], in[9], in[10]}, {in[11], in[12], in[13]}};
    const double ext[3] = {in[14], in[15], in[16]};
    double lm[2][10];
    for (int l = 0; l < 2; ++l) for (int k = 0; k < 10; ++k) lm[l][k] = lmf[10 * l + k];
    double lrho[2], lj[2][3], lg[2][3], lG;
    flbm::adj_modes<double>(rho, j, g, ext, G, lm, lrho, lj, lg, lG);
    out[0] = lrho[0]; out[1] = lrho[1];
    for (int l = 0; l < 2; ++l) for (int a = 0; a < 3; ++a) { out[2 + 3 * l + a] = lj[l][a]; out[8 + 3 * l + a] = lg[l][a]; }
    out[14] = lG;
}
extern "C" void adj_ab(const double* in, double G, const double* ab, double* out) {
    const double rho[2] = {in[0], in[1]};
    const double j[2][3] = {{in[2], in[3], in[4]}, {in[5], in[6], in[7]}};
    const double g[2][3] = {{in[8], in[9], in[10]}, {in[11], in[12], in[13]}};
    const double ext[3] = {in[14], in[15], in[16]};
    const double a[2] = {ab[0], ab[1]};
    const double b[2][3] = {{ab[2], ab[3], ab[4]}, {ab[5], ab[6], ab[7]}};
    double lrho[2], lj[2][3], lg[2][3], lG;
    flbm::adj_modes_ab<double>(rho, j, g, ext, G, a, b, lrho, lj, lg, lG);
    out[0] = lrho[0]; out[1] = lrho[1];
    for (int l = 0; l < 2; ++l) for (int c = 0; c < 3; ++c) { out[2 + 3 * l + c] = lj[l][c]; out[8 + 3 * l + c] = lg[l][c]; }
    out[14] = lG;
}
"""


@pytest.fixture(scope="module")
def shim(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("adjmath")
    src = d / "shim.cpp"
    src.write_text(SHIM)
    lib = d / "libshim.so"
    subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-I", CSRC, "-o", str(lib), str(src)], check=True)
    L = ctypes.CDLL(str(lib))
    dp = ctypes.POINTER(ctypes.c_double)
    L.fwd.argtypes = [dp, ctypes.c_double, dp]
    L.adj.argtypes = [dp, ctypes.c_double, dp, dp]
    L.adj_ab.argtypes = [dp, ctypes.c_double, dp, dp]
    L.adj_ab_df.argtypes = [dp, ctypes.c_double, dp, dp]
    fp = ctypes.POINTER(ctypes.c_float)
    L.adj_ab_mixed.argtypes = [fp, ctypes.c_float, dp, ctypes.c_int, dp]
    L.df_op.argtypes = [ctypes.c_int, fp, fp, fp]
    return L


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _fwd(L, x, G):
    ms = np.zeros(20)
    L.fwd(_p(np.ascontiguousarray(x)), G, _p(ms))
    return ms


@pytest.mark.parametrize("seed", range(6))
def test_adjoint_is_jacobian_transpose(shim, seed):
    rng = np.random.default_rng(seed)
    x = np.concatenate([[1.0 + 0.1 * rng.standard_normal(), 0.05 + 0.01 * rng.standard_normal()],
                        0.05 * rng.standard_normal(6), 0.1 * rng.standard_normal(6),
                        (1e-3 * rng.standard_normal(3)) if seed % 2 else np.zeros(3)])
    G = 1.2 + 0.3 * rng.standard_normal()
    lm = rng.standard_normal(20)
    out = np.zeros(15)
    shim.adj(_p(x), G, _p(lm), _p(out))
    v = rng.standard_normal(17)
    v[14:] = 0.0  # ext is a constant, not an input
    vG = rng.standard_normal()
    h = 1e-5
    jv = (_fwd(shim, x + h * v, G + h * vG) - _fwd(shim, x - h * v, G - h * vG)) / (2 * h)
    lhs = lm @ jv
    rhs = out[:14] @ v[:14] + out[14] * vG
    assert abs(lhs - rhs) <= 1e-8 * max(1.0, abs(lhs))


def test_modes_at_rest_are_the_equilibrium(shim):
    """Zero momentum and force: m*_0 = rho_l, every other mode 0 (the rest
    state of Section 2's collision)."""
    x = np.zeros(17)
    x[0], x[1] = 1.0, 0.05
    ms = _fwd(shim, x, 1.2)
    assert ms[0] == 1.0 and ms[10] == 0.05
    assert np.all(ms[1:10] == 0.0) and np.all(ms[11:20] == 0.0)


@pytest.mark.parametrize("seed", range(4))
def test_density_momentum_part_equals_the_general_transpose(shim, seed):
    """adj_modes_ab(a, b) = adj_modes with m*_0 = a, m*_1..3 = b, other modes 0."""
    rng = np.random.default_rng(100 + seed)
    x = np.concatenate([[1.0, 0.05], 0.05 * rng.standard_normal(6), 0.1 * rng.standard_normal(6),
                        1e-3 * rng.standard_normal(3)])
    ab = rng.standard_normal(8)
    lm = np.zeros(20)
    lm[0], lm[10] = ab[0], ab[1]
    lm[1:4], lm[11:14] = ab[2:5], ab[5:8]
    o1, o2 = np.zeros(15), np.zeros(15)
    shim.adj(_p(x), 1.3, _p(lm), _p(o1))
    shim.adj_ab(_p(x), 1.3, _p(ab), _p(o2))
    assert np.allclose(o1, o2, rtol=1e-13, atol=1e-15)


def _split(v):
    hi = np.float32(v)
    return np.array([hi, np.float32(v - float(hi))], dtype=np.float32)


@pytest.mark.parametrize("op", range(6))
def test_double_float_operations_against_exact_arithmetic(shim, op):
    """Sum, difference, product and quotient of double-float numbers, and
    the sum and product of a double-float and a float, agree with the exact
    rational result of the represented values to 2^-44 relative (about
    48-bit operands)."""
    from fractions import Fraction

    rng = np.random.default_rng(7 + op)
    fp = ctypes.POINTER(ctypes.c_float)
    worst = 0.0
    for _ in range(2000):
        a = _split(rng.standard_normal() * 10.0 ** rng.integers(-3, 4))
        b = _split(rng.standard_normal() * 10.0 ** rng.integers(-3, 4))
        if op == 1:  # differences of close numbers: the adjoint's use
            b = _split(float(a[0]) * (1 + 1e-3 * rng.standard_normal()))
        if op >= 4:  # the second operand is a float
            b[1] = np.float32(0.0)
        out = np.zeros(2, dtype=np.float32)
        shim.df_op(op, a.ctypes.data_as(fp), b.ctypes.data_as(fp), out.ctypes.data_as(fp))
        fa = Fraction(float(a[0])) + Fraction(float(a[1]))
        fb = Fraction(float(b[0])) + Fraction(float(b[1]))
        exact = [fa + fb, fa - fb, fa * fb, fa / fb, fa + fb, fa * fb][op]
        got = Fraction(float(out[0])) + Fraction(float(out[1]))
        scale = [max(abs(fa), abs(fb)), max(abs(fa), abs(fb)), abs(exact), abs(exact),
                 max(abs(fa), abs(fb)), abs(exact)][op]
        worst = max(worst, float(abs(got - exact) / scale))
    assert worst <= 2.0 ** -44, worst


@pytest.mark.parametrize("seed", range(4))
def test_density_momentum_part_in_double_float(shim, seed):
    """adj_modes_ab in double-float arithmetic equals its double evaluation to
    1e-12 of the largest adjoint input (the large parts it carries)."""
    rng = np.random.default_rng(200 + seed)
    x = np.concatenate([[1.0 + 0.05 * rng.standard_normal(), 0.05 + 0.01 * rng.standard_normal()],
                        0.02 * rng.standard_normal(6), 0.1 * rng.standard_normal(6), 1e-4 * rng.standard_normal(3)])
    x = np.array([float(np.float32(v)) for v in x])  # the kernels' inputs are float
    ab = 1e3 * (1.0 + 0.01 * rng.standard_normal(8))
    o1, o2 = np.zeros(15), np.zeros(15)
    G = float(np.float32(1.2))
    shim.adj_ab(_p(x), G, _p(ab), _p(o1))
    shim.adj_ab_df(_p(x), G, _p(ab), _p(o2))
    assert np.max(np.abs(o1 - o2)) <= 1e-12 * np.max(np.abs(ab)), np.max(np.abs(o1 - o2))


@pytest.mark.parametrize("seed", range(4))
def test_mixed_density_momentum_part_in_double_float(shim, seed):
    """adj_modes_ab_mixed (float coefficients, double-float adjoint values)
    equals its evaluation with the same float coefficients and double adjoint
    values to 1e-12 of the largest adjoint input, and the double-float
    adj_modes_ab with exact coefficients to the float rounding of the
    coefficients (1e-6 of the largest adjoint input)."""
    rng = np.random.default_rng(300 + seed)
    x = np.concatenate([[1.0 + 0.05 * rng.standard_normal(), 0.05 + 0.01 * rng.standard_normal()],
                        0.02 * rng.standard_normal(6), 0.1 * rng.standard_normal(6), 1e-4 * rng.standard_normal(3)])
    xf = x.astype(np.float32)
    x = xf.astype(np.float64)
    ab = 1e3 * (1.0 + 0.01 * rng.standard_normal(8))
    G = np.float32(1.2)
    fp = ctypes.POINTER(ctypes.c_float)
    o_df, o_d, o_exact = np.zeros(15), np.zeros(15), np.zeros(15)
    shim.adj_ab_mixed(xf.ctypes.data_as(fp), ctypes.c_float(G), _p(ab), 1, _p(o_df))
    shim.adj_ab_mixed(xf.ctypes.data_as(fp), ctypes.c_float(G), _p(ab), 0, _p(o_d))
    shim.adj_ab(_p(x), float(G), _p(ab), _p(o_exact))
    scale = np.max(np.abs(ab))
    assert np.max(np.abs(o_df - o_d)) <= 1e-12 * scale, np.max(np.abs(o_df - o_d))
    assert np.max(np.abs(o_df - o_exact)) <= 1e-6 * scale, np.max(np.abs(o_df - o_exact))
