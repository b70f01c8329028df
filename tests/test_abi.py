"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function include/mwax.h declares; host-only entry points work on the CPU."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "mwax.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mwax_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("mwax_plan", "mwax_correlate", "mwax_destroy", "mwax_baseline_index",
              "mwax_plan_batch", "mwax_correlate_batch", "mwax_calib_loss", "mwax_calib_grad"):
        assert n in names


def test_library_exports_every_declared_symbol(mwax_lib):
    lib = ctypes.CDLL(mwax_lib.LIB_PATH)
    for n in declared_functions():
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", mwax_lib.LIB_PATH], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r"\bT (mwax_[a-z_]+)\b", out))
    assert set(declared_functions()) <= exported
    assert set(mwax_lib.SIGNATURES) == set(declared_functions())


def test_host_helpers(mwax_lib):
    mw = mwax_lib
    assert mw.n_baselines(512) == 131328
    assert mw.n_baselines(1024) == 524800
    assert mw.baseline_index(3, 1) == 7
    assert mw.baseline_index(1, 3) == -1
    for b in (0, 1, 2, 7, 524799, 131327):
        i, j = mw.baseline_pair(b)
        assert mw.baseline_index(i, j) == b and 0 <= j <= i
    assert mw.max_n_time(8) == 66572
    assert mw.max_n_time(4) == 21913098
    assert mw.max_n_time(5) == -1


def test_plan_rejects_bad_jobs_before_touching_the_device(mwax_lib):
    """Argument and int32-bound checks happen before any CUDA call, so they
    return their status on a machine without a GPU."""
    mw = mwax_lib
    L = mw.lib()
    h = ctypes.c_void_p()

    def plan(**kw):
        j = mw._job(**kw)
        return L.mwax_plan(ctypes.byref(h), ctypes.byref(j), None)

    assert plan(n_inputs=4, n_chan=1, n_time=66573, sample_bits=8) == 3  # OVERFLOW_BOUND
    assert plan(n_inputs=0, n_chan=1, n_time=10, sample_bits=8) == 1
    # empty integrations and empty bands are rejected, not planned
    assert plan(n_inputs=4, n_chan=0, n_time=10, sample_bits=8) == 1
    assert plan(n_inputs=4, n_chan=1, n_time=0, sample_bits=4) == 1
    assert plan(n_inputs=-2, n_chan=1, n_time=10, sample_bits=4) == 1
    assert plan(n_inputs=4, n_chan=1, n_time=10, sample_bits=6) == 1
    assert plan(n_inputs=4, n_chan=1, n_time=10, sample_bits=4, kind=1) == 4  # FP16 needs 8-bit
    assert L.mwax_plan(None, None, None) == 1
    assert h.value is None
    assert L.mwax_destroy(None) == 0


def test_grid_plan_rejects_bad_arguments_without_a_device(mwax_lib):
    """Argument checks run before any CUDA call: odd or tiny grids, too few
    tiles, non-positive cell size or width are INVALID_ARG (1)."""
    import ctypes

    import numpy as np

    L = mwax_lib.lib()
    xy = np.zeros((4, 2), np.float64)
    h = ctypes.c_void_p()
    cases = [(4, 8, 150e6, 1e6, 33, 1.0, 7, 1.0), (1, 8, 150e6, 1e6, 32, 1.0, 7, 1.0),
             (4, 8, 150e6, 1e6, 32, 0.0, 7, 1.0), (4, 8, 150e6, 1e6, 32, 1.0, 7, 0.0),
             (4, 0, 150e6, 1e6, 32, 1.0, 7, 1.0), (4, 8, 150e6, 1e6, 32, 1.0, 0, 1.0)]
    for nt, nc, f0, df, Ng, du, W, sg in cases:
        assert L.mwax_grid_plan(ctypes.byref(h), xy.ctypes.data, nt, nc, f0, df, Ng, du, W, sg,
                                None) == 1
    assert L.mwax_grid(None, None, None) == 1
    assert L.mwax_grid_destroy(None) == 1


@pytest.mark.parametrize("n_tiles,n_chan", [(1, 1), (1, 5), (2, 1), (2, 768), (3, 7), (5, 4),
                                            (8, 3), (9, 2), (17, 2)])
def test_pair_work_list_covers_every_tile_pair_once(mwax_lib, n_tiles, n_chan):
    """The pair mode's host-built work list: every tile pair I >= J of every
    channel appears exactly once; shared items are (I, J), (I, J+1) with
    J+1 <= I in one channel; two-diagonal items pair diagonals of the same or
    the next channel; single items are diagonals; channels appear in order."""
    mw = mwax_lib
    items = mw.pair_work_list(n_tiles, n_chan)
    seen = {}
    last_c = -1
    for typ, c0, I0, J0, c1, I1, J1 in items.tolist():
        assert c0 >= last_c
        last_c = c0
        if typ == 1:
            assert c1 == c0 and I1 == I0 and J1 == J0 + 1 and J1 <= I0
            pairs = [(c0, I0, J0), (c0, I0, J1)]
        elif typ == 2:
            assert I0 == J0 and I1 == J1 and c1 in (c0, c0 + 1)
            pairs = [(c0, I0, I0), (c1, I1, I1)]
        else:
            assert typ == 0 and I0 == J0
            pairs = [(c0, I0, J0)]
        for q in pairs:
            seen[q] = seen.get(q, 0) + 1
    want = {(c, I, J) for c in range(n_chan) for I in range(n_tiles) for J in range(I + 1)}
    assert set(seen) == want and all(v == 1 for v in seen.values())
    # work balance: every item but at most one holds two tile pairs
    assert (items[:, 0] == 0).sum() <= 1
    assert mw.lib().mwax_pair_work_list(0, 1, None, 0) == -1
    assert mw.lib().mwax_pair_work_list(256, 1, None, 0) == -1


def test_calib_workspace_sizes(mwax_lib):
    """Workspace sizes from the partial-sum layout: per (32 x 32 input tile,
    channel group or channel) a row and a column complex partial per input,
    loss partials, and for the solves a real den partial per row and column;
    -1 for shapes out of range."""
    L = mwax_lib.lib()
    N, C = 1024, 768
    tiles = 32 * 33 // 2
    slots = tiles * C * 32
    loss_bytes = -(-tiles * (C // 8) * 4 // 256) * 256
    assert L.mwax_calib_chan_workspace_bytes(N, C) == slots * 16 + loss_bytes
    assert L.mwax_calib_chan_solve_workspace_bytes(N, C) == slots * 24 + loss_bytes
    assert L.mwax_calib_workspace_bytes(N, C) > 0
    for n, c in ((1, 4), (2, 0), (65537, 1), (4, 65535 * 8 + 1)):
        assert L.mwax_calib_chan_workspace_bytes(n, c) == -1
        assert L.mwax_calib_chan_solve_workspace_bytes(n, c) == -1
    assert L.mwax_calib_chan_workspace_bytes(2, 65535 * 8) > 0


def _build_c_client(mw, tmp_path):
    import shutil
    import subprocess

    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    lib_dir = os.path.dirname(mw.LIB_PATH)
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    cuda_lib = next((d for d in (os.path.join(cuda, "lib64"), os.path.join(cuda, "lib"))
                     if os.path.isdir(d)), os.path.join(cuda, "lib64"))
    exe = str(tmp_path / "abi_client")
    subprocess.run([gcc, "-std=c11", "-Wall", "-Werror", "-I", os.path.join(root, "include"),
                    "-I", os.path.join(cuda, "include"),
                    os.path.join(root, "tests", "c_client", "abi_client.c"),
                    "-L", lib_dir, "-lmwax", "-Wl,-rpath," + lib_dir,
                    "-L", cuda_lib, "-lcudart", "-Wl,-rpath," + cuda_lib, "-o", exe], check=True)
    case = os.path.join(root, "tests", "golden", "c_client_corr.txt")
    return exe, case


def _run_c_client(exe, case):
    import subprocess

    out = subprocess.run([exe, case], check=True, capture_output=True, text=True).stdout
    return dict(line.split(" ", 1) for line in out.strip().splitlines())


def test_plain_c_client_builds_and_runs(mwax_lib, tmp_path):
    """The boundary is a C library: a plain C program compiled against
    include/mwax.h (gcc, C11) links libmwax.so and gets the host-only answers
    (baseline helpers, the int32 bound, a refused plan, the pair-mode work
    list) without Python or torch."""
    exe, case = _build_c_client(mwax_lib, tmp_path)
    got = _run_c_client(exe, case)
    assert got["n_baselines_512"] == "131328"
    assert got["n_baselines_1024"] == "524800"
    assert got["baseline_index_5_3"] == "18"
    assert got["baseline_pair_status"] == "0" and got["baseline_pair_18"] == "5 3"
    assert got["max_n_time_8"] == "66572" and got["max_n_time_4"] == "21913098"
    assert got["plan_overflow_status"] == "3"
    assert got["plan_overflow_string"]
    assert got["work_list_tile_pairs"] == str(2 * 36)
    assert int(got["work_list_items"]) == 36  # 2 x 36 pairs, two per item
    assert got["calib_jones_ws_odd"] == "-1"


@pytest.mark.gpu
def test_plain_c_client_correlates_on_the_device(mwax_lib, tmp_path):
    """The same C program on a GPU: plan, correlate with device buffers and
    with host buffers, destroy -- every visibility equal to the oracle's
    (stored by tests/golden/make_c_client_golden.py)."""
    exe, case = _build_c_client(mwax_lib, tmp_path)
    got = _run_c_client(exe, case)
    assert "device_skipped" not in got
    assert got["plan_status"] == "0" and got["correlate_status"] == "0"
    assert got["plan_device_status"] == "0" and got["correlate_host_status"] == "0"
    assert got["destroy_status"] == "0"
    assert int(got["values_compared"]) == 2 * 20 * 21
    assert got["device_mismatches"] == "0" and got["host_mismatches"] == "0"
