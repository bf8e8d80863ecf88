"""Host-side checks of the C ABI: the library builds for sm_103a, loads, exports
every function include/fmm.h declares, validates arguments before touching a
device, sizes workspaces, and refuses to compute without a GPU (no CPU path)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def F():
    from paper_1205_2927_gb300 import build
    build.build()
    from paper_1205_2927_gb300 import fmm
    return fmm


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(fmm_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_every_declared_symbol_is_exported(F):
    names = declared_functions()
    assert "fmm_plan" in names and "fmm_gemm" in names and "fmm_gemm_batched" in names and "fmm_free" in names
    lib = C.CDLL(F._build.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_every_declared_symbol_has_a_binding(F):
    # the binding carries the C-ABI's names (argument marshalling only)
    missing = [n for n in declared_functions() if not callable(getattr(F, n, None))]
    assert not missing, missing
    o = F.fmm_options_default()
    assert (o.depth, o.cutoff) == (-1, 2048)
    assert F.fmm_status_string(7) == "FMM_ERR_TIMEOUT"


def test_options_default(F):
    o = F.options()
    assert (o.depth, o.cutoff, o.leaf_tile, o.precision, o.odd, o.planner, o.algo) == (-1, 2048, 0, 0, 3, 0, 0)


def test_status_strings(F):
    lib = F.library()
    for code, name in F.STATUS_NAMES.items():
        assert lib.fmm_status_string(code).decode() == name


def _query(F, M, N, K, **kw):
    return F.fmm_plan(M, N, K, max(K, 1), max(N, 1), max(N, 1), F.options(**kw), query_only=True)[1]


def test_workspace_query_grows_with_depth(F):
    n = 4096
    sizes = [_query(F, n, n, n, depth=d) for d in range(5)]
    assert all(s > 0 and s % 256 == 0 for s in sizes)
    assert sizes[1] < sizes[2] < sizes[3] < sizes[4]
    # depth 1: 7 child operands per side (n/2)^2 each, 7 products (n/2)^2
    q = (n // 2) ** 2 * 4
    assert sizes[1] >= 21 * q


@pytest.mark.parametrize("n,d,prec,es", [(16384, 3, "fp32", 4), (16384, 2, "fp32", 4), (8192, 3, "bf16x3", 2),
                                          (4096, 0, "fp32", 4)])
def test_workspace_closed_forms(F, n, d, prec, es):
    # the split planes (hi and lo, both sides, every leaf) plus the leaf
    # products are the whole workspace, apart from the status word and the
    # tile-scheduling area (< 256 KB): no transposed copies or middle levels
    # (the unfused last level: fuse_last = -1; the fused layout has its own test)
    need = _query(F, n, n, n, depth=d, precision=prec, leaf_tile=512, fuse_last=-1)
    leaves, h = 7 ** d, n >> d
    planes = 2 * 2 * leaves * h * h * es
    products = leaves * h * h * 4 if d > 0 else 0
    assert 0 <= need - planes - products < 256 * 1024, need - planes - products


def test_workspace_query_pads_to_level_granule(F):
    # 1000 at depth 2 pads to a multiple of 16: 1008
    s = _query(F, 1000, 1000, 1000, depth=2)
    s_exact = _query(F, 1008, 1008, 1008, depth=2)
    assert s == s_exact


@pytest.mark.parametrize("args", [
    (-1, 4, 4, 4, 4, 4), (4, 4, 4, 3, 4, 4), (4, 4, 4, 4, 3, 4), (4, 4, 4, 4, 4, 3),
])
def test_invalid_sizes_rejected(F, args):
    need = C.c_size_t(0)
    st = F.library().fmm_plan(None, *args, None, None, 0, C.byref(need), None)
    assert st == 1  # FMM_ERR_INVALID_ARG


def test_invalid_options_rejected(F):
    need = C.c_size_t(0)
    lib = F.library()
    for kw in ({"leaf_tile": 64}, {"depth": 9}, {"precision": 7}):
        o = F.options(**kw)
        assert lib.fmm_plan(None, 64, 64, 64, 64, 64, 64, C.byref(o), None, 0, C.byref(need), None) == 1


def test_gemm_rejects_null_plan(F):
    assert F.library().fmm_gemm(None, C.c_float(1), None, None, C.c_float(0), None, None) == 1
    F.library().fmm_free(None)  # NULL-safe
    assert F.library().fmm_plan_phase_bytes(None, None, None) == 1
    assert F.library().fmm_wait_selftest(None, 20_000_000, None) == 1


def test_no_cpu_fallback_without_gpu(F):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    need = C.c_size_t(0)
    o = F.options(depth=0)
    st = F.library().fmm_plan(C.byref(h), 64, 64, 64, 64, 64, 64, C.byref(o), None, 0, C.byref(need), None)
    assert st == 8  # FMM_ERR_NO_DEVICE
    assert not h.value


def test_peel_workspace_has_no_padding(F):
    # peel: the recursion covers the even core only; pad rounds the sizes up
    s_peel = _query(F, 1000, 1000, 1000, depth=3, odd="peel")
    s_pad = _query(F, 1000, 1000, 1000, depth=3, odd="pad")
    s_core = _query(F, 992, 992, 992, depth=3, odd="pad")
    assert s_peel > s_core        # core buffers + transposed B and aligned A for the border
    assert s_pad > s_core         # 1000 -> 1024


def test_plan_features_and_cost_model_file(F, tmp_path):
    import numpy as np
    from paper_1205_2927_gb300 import planner as PL
    assert F.fmm_plan_features(4096, 2048, 1024, 2, 256, 1) == [12.0, 10.0, 11.0, 2.0, 2.0, 1.0]
    p = PL.init_params(3)
    assert p.shape == (F.NPARAM,)
    PL.save(tmp_path / "m.bin", p, np.arange(6), np.ones(6))
    q, mean, std = PL.load(tmp_path / "m.bin")
    assert np.array_equal(q, p) and np.array_equal(mean, np.arange(6)) and np.all(std == 1)


def test_cost_model_registration_validates(F):
    import ctypes
    lib = F.library()
    P = (ctypes.c_float * F.NPARAM)()
    m = (ctypes.c_float * 6)()
    bad = (ctypes.c_float * 6)(*([1.0] * 5 + [0.0]))
    assert lib.fmm_set_cost_model(P, m, bad) == 1
    assert lib.fmm_set_cost_model(None, None, None) == 0


def test_exhaustive_query_includes_scratch(F):
    fixed = _query(F, 2048, 2048, 2048, planner="fixed", depth=1)
    ex = _query(F, 2048, 2048, 2048, planner="exhaustive")
    assert ex > fixed + 3 * 2048 * 2048 * 4 - 1


def test_classical_recursion_options(F):
    # Table 1's recursion reuses the depth-0 operands: the same workspace at every depth
    n = 2048
    sizes = [_query(F, n, n, n, depth=d, algo="classical") for d in range(4)]
    assert sizes[0] == _query(F, n, n, n, depth=0)
    assert len(set(sizes)) == 1
    need = C.c_size_t(0)
    lib = F.library()
    o = F.options(algo="classical", host_operands=1)
    assert lib.fmm_plan(None, 64, 64, 64, 64, 64, 64, C.byref(o), None, 0, C.byref(need), None) == 6


def test_static_wrapper_rejects_bad_operands_before_any_call(F, monkeypatch):
    torch = pytest.importorskip("torch")

    class NoCall:
        def __getattr__(self, name):
            raise AssertionError(f"the library was called ({name}) before the operand checks")

    monkeypatch.setattr(F, "_lib", NoCall())
    A = torch.zeros(8, 6)
    B = torch.zeros(6, 5)
    cases = [
        (A, torch.zeros(5, 5), torch.zeros(8, 5), ValueError, "rows"),       # B shorter than A's K
        (A, B, torch.zeros(7, 5), ValueError, "expected"),                   # C too small
        (A, B, torch.zeros(8, 4), ValueError, "expected"),
        (A, B.reshape(-1), torch.zeros(8, 5), ValueError, "2-D"),
        (A.double(), B, torch.zeros(8, 5), TypeError, "float32"),
        (A, B, torch.zeros(8, 5), ValueError, "CUDA"),                       # host tensors
    ]
    for a, b, c, exc, text in cases:
        with pytest.raises(exc, match=text):
            F.fmm_gemm_static(a, b, c)


def test_static_status_without_gpu_is_no_device(F):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    assert F.library().fmm_gemm_static_status(None) == 8


@pytest.mark.parametrize("n,d,prec,es", [(16384, 3, "fp32", 4), (8192, 2, "fp32", 4), (8192, 3, "fp16x3", 2),
                                          (8192, 4, "fp32", 4)])
def test_fused_workspace_closed_forms(F, n, d, prec, es):
    # fuse_last = 1: the split planes, the level-(d-1) node outputs (7^(d-1)
    # nodes of (2h)^2 floats, h the leaf size) and the running tiles of up to
    # 128 CTA pairs (512 KB each) replace the 7^d leaf products
    need = _query(F, n, n, n, depth=d, precision=prec, leaf_tile=512, fuse_last=1, odd="pad")
    leaves, h = 7 ** d, n >> d
    planes = 2 * 2 * leaves * h * h * es
    nodes = 7 ** (d - 1) * (2 * h) ** 2 * 4
    running = 128 * 2 * 2 * 128 * 256 * 4
    # depth 4 keeps the root level's 7 children per side (fp32); the bottom three
    # levels run as one pass
    root_children = 2 * 7 * (n // 2) ** 2 * 4 if d == 4 else 0
    rest = need - planes - nodes - running - root_children
    assert 0 <= rest < 256 * 1024, rest
    # the library's default fuses at depths 2 and 3 only
    default = _query(F, n, n, n, depth=d, precision=prec, leaf_tile=512, odd="pad")
    assert default == (need if d <= 3 else _query(F, n, n, n, depth=d, precision=prec, leaf_tile=512,
                                                  fuse_last=-1, odd="pad"))
    # by default only where the leaves are whole 256 x 256 tiles: n = 19000
    # (leaves 2376 wide at depth 3, 4752 at depth 2) stays unfused
    for dd in (2, 3):
        assert _query(F, 19000, 19000, 19000, depth=dd, precision=prec, leaf_tile=512, odd="pad") == \
            _query(F, 19000, 19000, 19000, depth=dd, precision=prec, leaf_tile=512, fuse_last=-1, odd="pad")
        assert _query(F, 19000, 19000, 19000, depth=dd, precision=prec, leaf_tile=512, fuse_last=1, odd="pad") != \
            _query(F, 19000, 19000, 19000, depth=dd, precision=prec, leaf_tile=512, fuse_last=-1, odd="pad")
    # options a fused plan cannot take fall back to the unfused schedule
    assert _query(F, n, n, n, depth=1, precision=prec, leaf_tile=512, fuse_last=1) == \
        _query(F, n, n, n, depth=1, precision=prec, leaf_tile=512, fuse_last=-1)
    assert _query(F, n, n, n, depth=d, precision="tf32", leaf_tile=512, fuse_last=1) == \
        _query(F, n, n, n, depth=d, precision="tf32", leaf_tile=512, fuse_last=-1)


def test_fuse_last_option_validated(F):
    need = C.c_size_t(0)
    for bad in (2, -2):
        o = F.options(fuse_last=bad)
        assert F.library().fmm_plan(None, 64, 64, 64, 64, 64, 64, C.byref(o), None, 0, C.byref(need), None) == 1


def test_host_copy_option_validated(F):
    # 0 library default, 1 copy engines, 2 SM loads/stores; anything else is rejected
    need = C.c_size_t(0)
    assert F.options().host_copy == 0
    for ok in (0, 1, 2):
        o = F.options(host_operands=1, host_copy=ok)
        assert F.library().fmm_plan(None, 64, 64, 64, 64, 64, 64, C.byref(o), None, 0, C.byref(need), None) == 0
    for bad in (3, -1):
        o = F.options(host_operands=1, host_copy=bad)
        assert F.library().fmm_plan(None, 64, 64, 64, 64, 64, 64, C.byref(o), None, 0, C.byref(need), None) == 1
    assert F.options(host_copy="sm").host_copy == 2 and F.options(host_copy="engine").host_copy == 1


def test_batched_planner_workspace_includes_scratch_outputs(F):
    # the exhaustive batched planner times whole-batch launches on scratch
    # outputs in the workspace: its query covers the fixed plan plus them
    shapes = [(512, 256, 384), (1024, 1024, 1024), (300, 700, 128)]
    n = len(shapes)
    i64 = C.c_int64 * n
    arrs = (i64(*[m for m, k, nn in shapes]), i64(*[nn for m, k, nn in shapes]), i64(*[k for m, k, nn in shapes]),
            None, i64(*[k for m, k, nn in shapes]), None, i64(*[nn for m, k, nn in shapes]), None,
            i64(*[nn for m, k, nn in shapes]), (C.c_float * n)(*[1.0] * n), (C.c_float * n)(*[0.0] * n))
    need = {}
    for pl in ("fixed", "exhaustive", "mlp"):
        o = F.options(planner=pl)
        sz = C.c_size_t(0)
        assert F.library().fmm_batched_plan(None, n, *arrs, C.byref(o), None, 0, C.byref(sz), None) == 0
        need[pl] = sz.value
    outputs = sum(m * nn * 4 for m, k, nn in shapes)
    assert need["exhaustive"] >= need["fixed"] + outputs
    assert need["mlp"] == need["exhaustive"]


@pytest.mark.parametrize("prec", ["fp32", "tf32", "bf16x3", "fp16x3"])
@pytest.mark.parametrize("planner", ["fixed", "exhaustive"])
def test_batched_size_query_with_null_operand_arrays(F, prec, planner):
    # the header allows A, B, C == NULL in a size query: no operand array is read
    shapes = [(100, 50, 60), (700, 640, 512), (16, 3000, 9)]
    n = len(shapes)
    i64 = C.c_int64 * n
    arrs = (i64(*[m for m, k, nn in shapes]), i64(*[nn for m, k, nn in shapes]), i64(*[k for m, k, nn in shapes]),
            None, i64(*[k for m, k, nn in shapes]), None, i64(*[nn for m, k, nn in shapes]), None,
            i64(*[nn for m, k, nn in shapes]), (C.c_float * n)(*[1.0] * n), (C.c_float * n)(*[0.0] * n))
    o = F.options(precision=prec, planner=planner, cutoff=64)
    sz = C.c_size_t(0)
    assert F.library().fmm_batched_plan(None, n, *arrs, C.byref(o), None, 0, C.byref(sz), None) == 0
    assert sz.value > 0


def test_tile_peel_workspace_covers_only_the_whole_tile_core(F):
    # FMM_ODD_TILE at depth 3 on pair tiles: the recursion covers
    # floor(n / 2048) * 2048 of M and N; n = 16640 -> a 16384 core (leaves of
    # 2048 = 8 whole tiles), so its planes are those of n = 16384 at K = 16640's
    # granule-32 core, with the border's B^T and A copies beside them
    tile = _query(F, 16640, 16640, 16640, depth=3, leaf_tile=512, odd="tile", fuse_last=-1)
    pad = _query(F, 16640, 16640, 16640, depth=3, leaf_tile=512, odd="pad", fuse_last=-1)
    leaves = 343
    planes = 2 * leaves * 2048 * 2080 * 4 * 2          # both sides, raw + lo, leaf K = 16640 / 8 = 2080
    products = leaves * 2048 * 2048 * 4
    border = 2 * 16640 * 16640 * 4                       # B^T and an aligned copy of A
    assert 0 <= tile - planes - products - border < 256 * 1024, tile - planes - products - border
    assert tile < pad + border


@pytest.mark.parametrize("n,d,resolved", [(16640, 3, "tile"), (16896, 3, "pad"), (19000, 3, "pad"),
                                          (20224, 2, "pad"), (16384, 3, "pad"), (18688, 3, "tile"),
                                          (8448, 3, "tile"), (10752, 3, "pad"), (9344, 2, "tile")])
def test_auto_odd_mode_resolution(F, n, d, resolved):
    # AUTO peels to whole leaf tiles when each remainder is at most an eighth of
    # the granule (256 * 2^d on CTA pairs), else pads: its workspace is that mode's
    auto = _query(F, n, n, n, depth=d, leaf_tile=512, odd="auto")
    want = _query(F, n, n, n, depth=d, leaf_tile=512, odd=resolved)
    assert auto == want


def test_auto_odd_mode_accepted_by_host_and_batched_plans(F):
    need = C.c_size_t(0)
    o = F.options(odd="auto", host_operands=1, depth=1)
    assert F.library().fmm_plan(None, 1000, 1000, 1000, 1000, 1000, 1000, C.byref(o), None, 0, C.byref(need), None) == 0
    o = F.options(odd="tile", host_operands=1, depth=1)
    assert F.library().fmm_plan(None, 1000, 1000, 1000, 1000, 1000, 1000, C.byref(o), None, 0, C.byref(need), None) == 6


def test_leading_dimension_of_empty_operands(F):
    # numpy-backed empty tensors carry stride 0; the binding passes a valid
    # leading dimension for them (they are never read), so a K = 0 member of a
    # batch is not refused for ld < N
    import numpy as np
    import torch
    assert F._ld(torch.from_numpy(np.zeros((0, 7), np.float32))) == 7
    assert F._ld(torch.from_numpy(np.zeros((5, 0), np.float32))) == 1
    assert F._ld(torch.zeros((4, 6))[:, :3]) == 6
