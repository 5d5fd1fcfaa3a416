"""C ABI: the library builds, loads and exports what include/ngdbf.h declares (no GPU needed)."""
import ctypes
import re

import numpy as np
import pytest

from paper_1402_2773_gb300 import _build, ngdbf


@pytest.fixture(scope="module")
def lib():
    _build.build_cuda()
    return ngdbf.load()


def test_header_declares_the_boundary():
    names = ngdbf.declared_functions()
    for want in ("ngdbf_code_create", "ngdbf_code_destroy", "ngdbf_decode", "ngdbf_decode_host",
                 "ngdbf_last_error", "ngdbf_code_info", "ngdbf_last_launch"):
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    for name in ngdbf.declared_functions():
        assert hasattr(lib, name), name


def test_params_struct_matches_header():
    src = open(ngdbf.HEADER).read()
    body = re.search(r"typedef struct ngdbf_params \{(.*?)\} ngdbf_params;", src, re.S).group(1)
    fields = re.findall(r"\b(float|int32_t)\s+([a-z_]+);", body)
    assert [f for _, f in fields] == ["w", "theta", "eta", "lambda", "y_max", "t_max", "smooth_window",
                                      "variant", "precision", "q_bits"]
    assert ctypes.sizeof(ngdbf.ngdbf_params) == 4 * len(fields)


def test_host_validation_without_a_device(lib):
    """Structural errors are reported before any CUDA call, with a message."""
    h = ctypes.c_void_p()
    i32p = ctypes.POINTER(ctypes.c_int32)

    def create(n, m, rp, ci):
        rp = np.ascontiguousarray(rp, np.int32)
        ci = np.ascontiguousarray(ci, np.int32)
        return lib.ngdbf_code_create(n, m, rp.ctypes.data_as(i32p), ci.ctypes.data_as(i32p), ctypes.byref(h))

    assert create(4, 4, [0, 1, 2, 3, 4], [0, 1, 2, 3]) == ngdbf.NGDBF_ERR_INVALID_ARG      # n > m
    assert create(4, 2, [0, 2, 4], [0, 5, 1, 2]) == ngdbf.NGDBF_ERR_INVALID_ARG            # index
    assert "range" in lib.ngdbf_last_error().decode()
    assert create(4, 2, [0, 2, 4], [0, 0, 1, 2]) == ngdbf.NGDBF_ERR_INVALID_ARG            # repeat
    assert create(4, 2, [0, 2, 2], [0, 1]) == ngdbf.NGDBF_ERR_INVALID_ARG                  # empty row
    assert create(4, 2, [0, 2, 3], [0, 1, 2]) == ngdbf.NGDBF_ERR_INVALID_ARG               # symbol 3 unused
    assert create(70000, 2, [0, 1, 2], [0, 1]) == ngdbf.NGDBF_ERR_UNSUPPORTED              # n too large
    p = ngdbf.make_params()
    assert lib.ngdbf_decode(None, None, 1, 0.5, ctypes.byref(p), 1, 0, None, None, None, None) == \
        ngdbf.NGDBF_ERR_INVALID_ARG
    assert lib.ngdbf_decode_host(None, None, 1, 0.5, ctypes.byref(p), 1, 0, None, None, None, 0) == \
        ngdbf.NGDBF_ERR_INVALID_ARG


def test_entry_points_check_arguments_before_any_device_call(lib):
    """Argument errors of the other entry points are reported with a status and a message,
    before any CUDA call (so they behave the same with or without a device)."""
    p = ngdbf.make_params()
    assert lib.ngdbf_decode_noalloc(None, None, 1, 0.5, ctypes.byref(p), 1, 0, None, None, None, None) == \
        ngdbf.NGDBF_ERR_INVALID_ARG
    assert lib.ngdbf_gaussian_range(0, 0, None, None) == ngdbf.NGDBF_OK            # nothing to do
    assert lib.ngdbf_gaussian_range(0, 4, None, None) == ngdbf.NGDBF_ERR_INVALID_ARG
    assert "NULL" in lib.ngdbf_last_error().decode()
    out = ctypes.c_void_p()
    for budget, inflight, jobs in ((0, 4, 16), (1 << 20, 0, 16), (1 << 20, 17, 16), (1 << 20, 4, 0),
                                   (1 << 20, 4, 5000)):
        assert lib.ngdbf_server_create(budget, inflight, jobs, 1, ctypes.byref(out)) == \
            ngdbf.NGDBF_ERR_INVALID_ARG
    assert lib.ngdbf_server_create(1 << 20, 4, 16, 1, None) == ngdbf.NGDBF_ERR_INVALID_ARG
    job = ngdbf.ngdbf_job()
    assert lib.ngdbf_batch_create(None, 0, 1, 0, None, ctypes.byref(out)) == ngdbf.NGDBF_ERR_INVALID_ARG
    assert lib.ngdbf_batch_create(ctypes.byref(job), 1, 1, 1 << 8, None, ctypes.byref(out)) == \
        ngdbf.NGDBF_ERR_INVALID_ARG
    assert "flags" in lib.ngdbf_last_error().decode()
    assert lib.ngdbf_batch_launch(None, None) == ngdbf.NGDBF_ERR_INVALID_ARG
    assert lib.ngdbf_server_wait(None, 1.0) == ngdbf.NGDBF_ERR_INVALID_ARG
    assert lib.ngdbf_code_destroy(None) == ngdbf.NGDBF_OK and lib.ngdbf_server_destroy(None) == ngdbf.NGDBF_OK


def test_missing_library_fails_loudly(tmp_path):
    with pytest.raises(RuntimeError, match="not built"):
        ngdbf.load(str(tmp_path / "absent.so"))


def test_struct_layouts_match_the_c_compiler(tmp_path):
    """sizeof/offsetof of every public struct, from gcc on include/ngdbf.h, equal the binding's."""
    import subprocess
    src = tmp_path / "layout.c"
    src.write_text('''#include <stddef.h>
#include <stdio.h>
#include "ngdbf.h"
#define F(T, f) printf("%s.%s %zu\\n", #T, #f, offsetof(T, f));
int main(void) {
    printf("ngdbf_params %zu\\nngdbf_job %zu\\nngdbf_launch_info %zu\\nngdbf_host_stats %zu\\n",
           sizeof(ngdbf_params), sizeof(ngdbf_job), sizeof(ngdbf_launch_info), sizeof(ngdbf_host_stats));
    F(ngdbf_host_stats, h2d_bytes) F(ngdbf_host_stats, h2d_ms) F(ngdbf_host_stats, wall_ms)
    F(ngdbf_job, code) F(ngdbf_job, y) F(ngdbf_job, n_frames) F(ngdbf_job, sigma) F(ngdbf_job, params)
    F(ngdbf_job, frame_offset) F(ngdbf_job, bits) F(ngdbf_job, iters) F(ngdbf_job, pass)
    F(ngdbf_params, q_bits) F(ngdbf_launch_info, sm_count) F(ngdbf_launch_info, tables_in_smem)
    return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", str(ngdbf.os.path.dirname(ngdbf.HEADER)), "-o", str(exe), str(src)])
    got = dict(ln.split() for ln in subprocess.check_output([str(exe)], text=True).splitlines())
    assert int(got["ngdbf_params"]) == ctypes.sizeof(ngdbf.ngdbf_params)
    assert int(got["ngdbf_job"]) == ctypes.sizeof(ngdbf.ngdbf_job)
    assert int(got["ngdbf_launch_info"]) == ctypes.sizeof(ngdbf.ngdbf_launch_info)
    assert int(got["ngdbf_host_stats"]) == ctypes.sizeof(ngdbf.ngdbf_host_stats)
    for f in ("h2d_bytes", "h2d_ms", "wall_ms"):
        assert int(got[f"ngdbf_host_stats.{f}"]) == getattr(ngdbf.ngdbf_host_stats, f).offset, f
    for f in ("code", "y", "n_frames", "sigma", "params", "frame_offset", "bits", "iters"):
        assert int(got[f"ngdbf_job.{f}"]) == getattr(ngdbf.ngdbf_job, f).offset, f
    assert int(got["ngdbf_job.pass"]) == ngdbf.ngdbf_job.pass_.offset
    assert int(got["ngdbf_params.q_bits"]) == ngdbf.ngdbf_params.q_bits.offset
    assert int(got["ngdbf_launch_info.sm_count"]) == ngdbf.ngdbf_launch_info.sm_count.offset
    assert int(got["ngdbf_launch_info.tables_in_smem"]) == ngdbf.ngdbf_launch_info.tables_in_smem.offset


def test_generator_table_equals_the_reference_and_an_independent_derivation():
    """The library's inverse-CDF table (host code of libngdbf.so, no GPU needed) equals the reference
    decoder's word for word, and an independent derivation -- scipy's ndtri at the Chebyshev
    points, cubic by a float64 Vandermonde solve -- agrees within one FP32 ulp on every coefficient
    (c3 carries the cancellation of a third difference: its FP32 word may differ by an ulp between
    double-precision routes, which is why the table is defined by one fixed double computation)."""
    import numpy as np
    from scipy.special import ndtri

    import oracle
    lib_tab = ngdbf.ngdbf_generator_table()
    ref_tab = oracle.load().icdf_table()
    assert lib_tab.tobytes() == ref_tab.tobytes()
    nodes = 0.5 * np.cos((2 * np.arange(4) + 1) * np.pi / 8)
    V = np.vander(nodes, 4, increasing=True)
    worst = 0.0
    for j in range(32):
        for s in range(8):
            g = ndtri(np.ldexp(8.0 + s + 0.5 + nodes, -(j + 5)))
            c = np.linalg.solve(V, g)
            w = lib_tab[j, s]
            ulp = np.spacing(np.abs(w)).astype(np.float64)
            worst = max(worst, float(np.max(np.abs(c - w.astype(np.float64)) / ulp)))
    assert worst <= 1.0, f"{worst:.2f} ulp"


def test_host_allocator_validation_without_a_device(lib):
    """ngdbf_host_alloc/free: argument errors and the huge-page size need no device."""
    p = ctypes.c_void_p()
    assert lib.ngdbf_host_alloc(0, ctypes.byref(p)) == ngdbf.NGDBF_ERR_INVALID_ARG
    assert lib.ngdbf_host_alloc(64, None) == ngdbf.NGDBF_ERR_INVALID_ARG
    assert lib.ngdbf_host_free(None) == ngdbf.NGDBF_OK
    buf = ctypes.create_string_buffer(64)
    assert lib.ngdbf_host_free(ctypes.addressof(buf)) == ngdbf.NGDBF_ERR_INVALID_ARG
    assert "ngdbf_host_alloc" in lib.ngdbf_last_error().decode()
    hp = ctypes.c_int64(-1)
    assert lib.ngdbf_host_huge_page_bytes(ctypes.byref(hp)) == ngdbf.NGDBF_OK
    try:
        want = int(open("/sys/kernel/mm/transparent_hugepage/hpage_pmd_size").read())
    except OSError:
        want = 0
    assert hp.value == want


def test_host_copy_mode_without_a_device(lib):
    m = ctypes.c_int32(-1)
    assert lib.ngdbf_get_host_copy_mode(ctypes.byref(m)) == ngdbf.NGDBF_OK
    assert m.value == ngdbf.NGDBF_HOST_COPY_STAGED              # the default
    assert lib.ngdbf_set_host_copy_mode(7) == ngdbf.NGDBF_ERR_INVALID_ARG
    assert lib.ngdbf_set_host_copy_mode(ngdbf.NGDBF_HOST_COPY_DIRECT) == ngdbf.NGDBF_OK
    assert lib.ngdbf_get_host_copy_mode(ctypes.byref(m)) == ngdbf.NGDBF_OK and m.value == ngdbf.NGDBF_HOST_COPY_DIRECT
    assert lib.ngdbf_set_host_copy_mode(ngdbf.NGDBF_HOST_COPY_STAGED) == ngdbf.NGDBF_OK
    assert lib.ngdbf_get_host_copy_mode(None) == ngdbf.NGDBF_ERR_INVALID_ARG
