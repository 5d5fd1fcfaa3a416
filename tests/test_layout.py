"""Shared-memory layouts (host side, no GPU): the per-job layouts that the job-table and serving
kernels compute for each code stay inside the launch's dynamic shared memory.

The serving kernel's shared memory is planned for the componentwise maxima (n, m, d_v, d_c) of
the codes of its kind, and each request is decoded in a layout of its own code within those
bytes: with its per-slot state when that fits, else without it.  The fallback must always fit
(a request of a smaller code never overruns the launch's bytes), and every layout must keep its
arrays 16-byte aligned, in order and inside its total.  The layout functions are host/device
functions of the kernel header; this test compiles them into a host program with nvcc.
"""
import os
import shutil
import subprocess

import pytest

from paper_1402_2773_gb300 import _build

SRC = r"""
#include "ngdbf_kernels.cuh"
#include <cstdio>
#include <cstdlib>
#include <cstdint>

using namespace ngdbf;

static uint64_t s = 0;
static uint32_t rnd() {            // splitmix64
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return (uint32_t)((z ^ (z >> 31)) >> 32);
}
static int in(int lo, int hi) { return lo + (int)(rnd() % (uint32_t)(hi - lo + 1)); }

static bool sane(const SmemLayout& L, const char* what) {
    const int32_t offs[] = {L.off_frame, L.off_start, L.off_ctl, L.off_best, L.off_trace, L.off_icdf,
                            L.off_cnt, L.off_xw, L.off_sw, L.off_thr, L.off_st, L.off_chk, L.off_sym};
    int32_t prev = -1;
    for (int32_t o : offs) {
        if (o == -1) continue;                              // array not placed
        if (o < 0 || o % 16 || o <= prev || o >= L.total) {
            printf("FAIL %s: offset %d (previous %d, total %d)\n", what, o, prev, L.total);
            return false;
        }
        prev = o;
    }
    return L.total % 16 == 0;
}

int main(int argc, char** argv) {
    s = strtoull(argv[1], nullptr, 10);
    const int cases = atoi(argv[2]);
    long fits_state = 0;
    for (int c = 0; c < cases; ++c) {
        const bool wide = rnd() & 1;
        const int Kn = in(8, 16384), Km = in(4, Kn), Kdv = wide ? in(8, 24) : in(1, 7), Kdc = in(2, 64);
        const int Kt = in(1, 500), P = in(0, 3);
        const bool adapt = rnd() & 1, st = rnd() & 1;
        // the kind's layout as the host plans it, with the placement it chose
        const SmemLayout K = smem_layout(Kn, Km, Kt, Kdv, Kdc, adapt, st, P, -1, wide ? 1 : 0);
        if (!sane(K, "kind")) return 1;
        for (int r = 0; r < 8; ++r) {
            const int n = in(1, Kn), m = in(1, Km), dv = wide ? in(8, Kdv) : in(1, Kdv), dc = in(1, Kdc);
            const int t = in(1, Kt);
            int tb = -1;
            // without state: always inside the kind's bytes
            const SmemLayout G = job_layout(n, m, t, dv, dc, adapt, false, wide, P, n, K.total, &tb);
            if (G.total > K.total || !sane(G, "job") || (tb & ~P)) {
                printf("FAIL job without state: n=%d m=%d dv=%d dc=%d: %d > %d bytes (kind n=%d m=%d dv=%d dc=%d)\n",
                       n, m, dv, dc, G.total, K.total, Kn, Km, Kdv, Kdc);
                return 1;
            }
            // with state: inside the kind's bytes whenever the kind's own layout holds the state
            const SmemLayout S = job_layout(n, m, t, dv, dc, adapt, true, wide, P, n, K.total, &tb);
            if (!sane(S, "job with state") || (st && S.total > K.total)) {
                printf("FAIL job with state: n=%d m=%d: %d > %d bytes\n", n, m, S.total, K.total);
                return 1;
            }
            fits_state += S.total <= K.total;
            // a code split over C CTAs holds at most ceil(n / C) symbols of state and counts
            const int C = 1 << in(1, 3);
            const int nl = (n + C - 1) / C;
            const SmemLayout Sp = job_layout(n, m, t, dv, dc, adapt, true, wide, P, nl, 1 << 30, &tb);
            const SmemLayout Su = job_layout(n, m, t, dv, dc, adapt, true, wide, P, n, 1 << 30, &tb);
            if (!sane(Sp, "split job") || Sp.total > Su.total) {
                printf("FAIL split job: n=%d C=%d: %d > %d bytes\n", n, C, Sp.total, Su.total);
                return 1;
            }
        }
    }
    printf("ok %d %ld\n", cases, fits_state);
    return 0;
}
"""


@pytest.fixture(scope="module")
def layout_prog(tmp_path_factory):
    nvcc = _build.nvcc()
    if shutil.which(nvcc) is None and not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("layout")
    src, exe = d / "layout_check.cu", d / "layout_check"
    src.write_text(SRC)
    subprocess.check_call([nvcc, "-std=c++17", "-O1", "-I", _build.CSRC, "-gencode", "arch=compute_103a,code=sm_103a",
                           "-o", str(exe), str(src)])
    return str(exe)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_job_layouts_fit_the_launch(layout_prog, seed):
    out = subprocess.run([layout_prog, str(seed), "4000"], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout + out.stderr
    tag, cases, with_state = out.stdout.split()
    assert tag == "ok" and int(cases) == 4000
    assert 0 < int(with_state) < 8 * 4000          # both outcomes occur: the state fits, or it does not
