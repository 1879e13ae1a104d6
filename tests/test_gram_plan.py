"""The Gram output plan (Eqs. rowB, rowC): which outputs each of a run's four
threads updates together with one packed FP32x2 operation, and from which
Delta elements.  Every output of every supported rank must be updated exactly
once, by a product of the right two elements (B_jk = d_j d_k, c_k = d_k x);
a dropped or doubled output, or a wrong operand, would silently corrupt B_i
or c_i.  The plan is plain constexpr C++, compiled here with the host compiler.
"""
import os
import shutil
import subprocess

import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1710_02261_gb300", "csrc")

PROG = r"""
#include <cstdio>
#include "gram_plan.cuh"
using namespace ptk;

template <int J> int check() {
    constexpr PackPlan<J> p{};
    constexpr Tri<J> tri;
    constexpr int NTRI = J * (J + 1) / 2, NOUT = NTRI + J;
    int seen[NOUT] = {};
    int bad = 0;
    for (int part = 0; part < 4; ++part) {
        if (p.np[part] > PackPlan<J>::PMAX) ++bad;
        for (int q = 0; q < p.np[part]; ++q) {
            const int g[2] = {p.g0[part][q], p.g1[part][q]};
            const int a[2] = {p.a0[part][q], p.a1[part][q]}, b[2] = {p.b0[part][q], p.b1[part][q]};
            if (g[0] < 0) ++bad;
            for (int u = 0; u < 2; ++u) {
                if (g[u] < 0) continue;
                if (g[u] >= NOUT) { ++bad; continue; }
                ++seen[g[u]];
                const int ea = g[u] < NTRI ? tri.j[g[u]] : g[u] - NTRI;
                const int eb = g[u] < NTRI ? tri.k[g[u]] : J;
                if (!((a[u] == ea && b[u] == eb) || (a[u] == eb && b[u] == ea))) ++bad;
            }
        }
    }
    for (int g = 0; g < NOUT; ++g) if (seen[g] != 1) ++bad;
    // the triangle enumeration itself: row-major over j <= k
    int q = 0;
    for (int j = 0; j < J; ++j)
        for (int k = j; k < J; ++k, ++q) {
            if (tri.j[q] != j || tri.k[q] != k) ++bad;
            if (PackPlan<J>::gtri(j, k) != q) ++bad;
        }
    if (bad) std::printf("J=%d: %d faults\n", J, bad);
    return bad;
}

int main() {
    int bad = check<1>() + check<2>() + check<3>() + check<4>() + check<5>() + check<6>() + check<7>() +
              check<8>() + check<9>() + check<10>() + check<11>() + check<12>() + check<13>() + check<14>() +
              check<15>() + check<16>();
    return bad ? 1 : 0;
}
"""


def test_pack_plan_covers_every_output_once(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "plan.cpp"
    src.write_text(PROG)
    exe = tmp_path / "plan"
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    run = subprocess.run([str(exe)], capture_output=True, text=True)
    assert run.returncode == 0, run.stdout
