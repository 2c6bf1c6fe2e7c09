"""Host-side checks of the C ABI (no GPU needed): the library loads, exports every symbol
include/*.h declare, validates plans before any CUDA call, and reports the output
shape of Eq. 2 (P0 x P1 x n0 x n1) and its workspace."""
import ctypes
import json
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in sorted(os.listdir(os.path.join(ROOT, "include")))
           if h.endswith(".h")]


@pytest.fixture(scope="module")
def nat():
    import __graft_entry__
    __graft_entry__._load_build_module().build()
    from paper_1707_08213_gb300 import _native
    return _native


def declared_functions():
    names = set()
    for h in HEADERS:
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"\b(swdft(?:2d|kd)_\w+)\s*\(", text))
    return sorted(names)


def test_header_declares_what_binding_lists(nat):
    assert sorted(nat.EXPORTS) == declared_functions()


def test_library_exports_every_declared_symbol(nat):
    lib = ctypes.CDLL(nat.LIB_PATH)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_version_and_status_strings(nat):
    assert nat.version() >= 200
    for code in range(-8, 1):
        assert nat.status_string(code).startswith("SWDFT_")
    assert "unknown" in nat.status_string(42)


def shp(N0, N1, n0, n1, **kw):
    d = dict(N0=N0, N1=N1, n0=n0, n1=n1)
    d.update(kw)
    return d


@pytest.mark.parametrize("shape,status", [
    (shp(16, 16, 5, 4), -2),           # neither a power of two nor 3^b 2^a
    (shp(16, 16, 4, 10), -2),
    (shp(16, 16, 4, 12), -4),          # binary column tree over mixed-radix row DFTs
    (shp(100, 100, 81, 3), -4),        # ternary trees are built up to 27
    (shp(120, 120, 96, 3), -4),        # mixed-radix trees up to 64
    (shp(40, 40, 16, 9), -4),          # binary column tree over ternary row DFTs
    (shp(40, 40, 8, 3), -4),
    (shp(16, 16, 32, 4), -3),          # window larger than the array
    (shp(16, 8, 4, 16), -3),
    (shp(0, 16, 1, 1), -1),            # empty array
    (shp(16, 16, 0, 4), -1),
    (shp(16, 16, 4, 4, ld=8), -1),     # row stride shorter than a row
    (shp(16, 16, 4, 4, dtype=7), -1),  # bad dtype
    (shp(16, 16, 4, 4, row_begin=5, row_end=3), -1),   # empty band
    (shp(16, 16, 4, 4, row_begin=0, row_end=14), -1),  # band past P0 = 13
    (shp(300, 300, 128, 4), -4),       # beyond the tree kernels' 64-point axis
])
def test_plan_validation(nat, shape, status):
    st, h = nat.raw_plan([shape], 0, 0, 1, 0)
    assert st == status
    assert h is None


def test_ternary_and_mixed_radix_windows_are_accepted_by_the_tree_only(nat):
    for n0, n1 in ((3, 3), (9, 27), (27, 1), (1, 9), (9, 16), (27, 64), (3, 2),
                   (6, 6), (12, 48), (54, 1), (1, 24), (18, 36), (48, 64), (36, 9)):
        st, h = nat.raw_plan([shp(60, 70, n0, n1)], 0, 0, 1, 0)
        assert st == 0, (n0, n1)
        nat.lib.swdft2d_destroy(h)
    assert nat.raw_plan([shp(40, 40, 27, 27)], 0, 0, 2, 0)[0] == -4   # tensor-core forms
    # a persistent batch runs ternary and mixed-radix arrays on their own launches
    for n0, n1 in ((9, 9), (12, 6)):
        st, h = nat.raw_plan([shp(40, 40, n0, n1), shp(40, 40, 8, 8)], 0, 0, 1, 4)
        assert st == 0
        nat.lib.swdft2d_destroy(h)
    p = nat.Plan([dict(N0=60, N1=70, n0=24, n1=12)])
    assert p.output_shape(0) == (37, 59, 24, 12)
    assert p.workspace_size() >= (16 + 37 + 23) * 59 * 12 * 8  # 2*n0/3 look-back rows
    p = nat.Plan([dict(N0=40, N1=70, n0=9, n1=27)])
    assert p.output_shape(0) == (32, 44, 9, 27)
    # z: 2*n0/3 look-back rows in front, then P0 + n0 - 1 rows of P1 * n1 complex64
    assert p.workspace_size() >= (6 + 32 + 8) * 44 * 27 * 8
    assert p.launch_count() == 2


def test_plan_validation_enums(nat):
    good = [shp(16, 16, 4, 4)]
    assert nat.raw_plan(good, 3, 0, 1, 0)[0] == -1      # norm
    assert nat.raw_plan(good, 0, 2, 1, 0)[0] == -1      # position convention
    assert nat.raw_plan(good, 0, 0, 9, 0)[0] == -1      # algorithm
    assert nat.raw_plan(good, 0, 0, 1, 1 << 9)[0] == -1  # unknown flag
    st, h = nat.raw_plan(good, 0, 0, 1, nat.FLAG_AUTOTUNE | nat.FLAG_GRAPH)  # tune on first execute
    assert st == 0
    nat.lib.swdft2d_destroy(h)
    assert nat.raw_plan([], 0, 0, 1, 0)[0] == -1          # empty batch
    st = nat.lib.swdft2d_plan(None, 1, None, 0, 0, 1, 0)
    assert st == -1


def test_adjoint_workspace_holds_z_and_the_chunk_side_rows(nat):
    """256x256 with 16x16 windows: the column adjoint splits 241 window rows into chunks of
    max(ceil(241/8), 6 n0) = 96 rows (3 chunks); each of the 2 boundaries keeps n0 - 1 side
    rows of P1*n1 complex64 after gz, which is z's size (n0/2 + 241 + n0 - 1 rows)."""
    p = nat.Plan([shp(256, 256, 16, 16)])
    r = lambda v: (v + 255) // 256 * 256
    z = (8 + 241 + 15) * 241 * 16 * 8
    side = 2 * 15 * 241 * 16 * 8
    assert p.workspace_size() == r(z) + r(side)
    assert p.launch_count(adjoint=True) == 3  # column pass, fold of the side rows, row pass


def test_output_shape_and_workspace(nat):
    p = nat.Plan([shp(64, 77, 8, 16), shp(33, 40, 32, 1, dtype=1)])
    assert p.output_shape(0) == (57, 62, 8, 16)
    assert p.output_shape(1) == (2, 40, 32, 1)
    # z workspace: (n0/2 padding + band rows + n0 - 1) x P1 x n1 complex64, largest array
    need = max((4 + 57 + 7) * 62 * 16 * 8, (16 + 2 + 31) * 40 * 1 * 8)
    ws = p.workspace_size()
    assert ws >= need and ws % 256 == 0
    with pytest.raises(nat.SwdftError):
        p.output_shape(2)
    p.destroy()


def test_band_in_both_position_conventions(nat):
    start = nat.Plan([shp(40, 20, 8, 4, row_begin=5, row_end=12)], pos="start")
    end = nat.Plan([shp(40, 20, 8, 4, row_begin=5 + 7, row_end=12 + 7)], pos="end")
    assert start.output_shape(0) == end.output_shape(0) == (7, 17, 8, 4)
    # row_end = 0: through the last window row
    tail = nat.Plan([shp(40, 20, 8, 4, row_begin=30, row_end=0)])
    assert tail.output_shape(0) == (3, 17, 8, 4)


def test_paper_output_size_example(nat):
    """Section 4.3: P0 = P1 = 400, n0 = n1 = 32 gives 163,840,000 coefficients."""
    with open(os.path.join(ROOT, "tests", "golden", "paper_printed_values.json")) as f:
        ex = json.load(f)["output_size_example"]
    N = ex["P0"] + ex["n0"] - 1
    p = nat.Plan([shp(N, N, ex["n0"], ex["n1"])])
    rows, P1, n0, n1 = p.output_shape(0)
    assert rows * P1 * n0 * n1 == ex["complex_numbers"]
    assert rows * P1 * n0 * n1 * ex["bytes_per_complex"] == ex["bytes"]


def test_execute_rejects_bad_buffers_before_cuda(nat):
    p = nat.Plan([shp(16, 16, 4, 4)])
    with pytest.raises(nat.SwdftError) as e:
        p.execute([0], [0], 0)
    assert e.value.status == -1
    with pytest.raises(nat.SwdftError) as e:
        p.execute([4096], [4096 + 8], 4096)   # output not 16-byte aligned
    assert e.value.status == -1
    with pytest.raises(nat.SwdftError) as e:
        p.execute([4096], [4096], 4096 + 64)  # workspace not 256-byte aligned
    assert e.value.status == -8
    with pytest.raises(nat.SwdftError) as e:
        p.execute_host([4096], [4096])        # plan made without SWDFT_FLAG_HOST_IO
    assert e.value.status == -1
    with pytest.raises(nat.SwdftError) as e:
        p.execute_stage(2, [4096], [4096], 4096)
    assert e.value.status == -1
    assert nat.lib.swdft2d_destroy(None) == 0


def test_launch_count(nat):
    # small windows use the fused form (one launch), larger ones two passes
    p = nat.Plan([shp(16, 16, 4, 4), shp(32, 32, 8, 8)])
    assert p.launch_count() == 2
    assert nat.Plan([shp(64, 64, 32, 32), shp(64, 64, 16, 64)]).launch_count() == 4
    # adjoint: column pass, the fold of the rows its chunks share, row pass
    assert nat.Plan([shp(64, 64, 4, 4)]).launch_count(adjoint=True) == 3
    assert nat.Plan([shp(18, 64, 4, 4)]).launch_count(adjoint=True) == 2  # one chunk: no fold


def test_twiddle_table_symmetry_via_plan(nat):
    # a plan of every supported length is accepted (FP64 twiddles built on the host)
    for m in range(0, 7):
        n = 1 << m
        p = nat.Plan([shp(n + 3, n + 5, n, n)])
        assert p.output_shape(0) == (4, 6, n, n)


# ------------------------------------------------------------------ k dimensions (swdftkd.h)

@pytest.mark.parametrize("N,n,kw,status", [
    ((), (), dict(k=0), -1),                          # no dimension
    ((4,) * 5, (1,) * 5, dict(k=5), -1),              # more than four
    ((8, 0, 8), (2, 1, 2), {}, -1),                   # empty extent
    ((8, 8, 8), (2, 0, 2), {}, -1),                   # empty window
    ((8, 8, 8), (2, 3, 2), {}, -2),                   # not a power of two
    ((8, 8, 8), (2, 16, 2), {}, -3),                  # window larger than the array
    ((200, 8, 8), (128, 2, 2), {}, -4),               # beyond the 64-point axis
    ((8, 8, 8), (2, 2, 2), dict(dtype=7), -1),        # bad dtype
    ((8, 8, 8), (2, 2, 2), dict(norm=3), -1),         # bad normalisation
    ((8, 8, 8), (2, 2, 2), dict(flags=1), -4),        # no flags for kD plans
])
def test_kd_plan_validation(nat, N, n, kw, status):
    st, h = nat.raw_plan_kd(N, n, **kw)
    assert st == status
    assert h is None


def test_kd_output_shape_workspace_and_launches(nat):
    N, n = (20, 24, 28), (4, 8, 2)
    p = nat.PlanKD(N, n)
    P = tuple(a - b + 1 for a, b in zip(N, n))
    assert p.output_shape() == P + n
    # z after the last dimension's levels: N0*N1 rows of P2*n2, with n1/2 look-back rows in
    # front; after dimension 1's levels: N0 rows of P1*n1*P2*n2 with n0/2 rows in front
    r = lambda b: (b + 255) // 256 * 256
    c2 = P[2] * n[2]
    c1 = P[1] * n[1] * c2
    assert p.workspace_size() == r(8 * (n[1] // 2 + N[0] * N[1]) * c2) + r(8 * (n[0] // 2 + N[0]) * c1)
    assert p.launch_count() == 3
    assert nat.PlanKD((5, 6, 7, 8), (2, 2, 4, 8)).launch_count() == 4
    # one and two dimensions run the 2D plan (two passes)
    assert nat.PlanKD((30,), (8,)).output_shape() == (23, 8)
    assert nat.PlanKD((30, 20), (8, 4)).output_shape() == (23, 17, 8, 4)
    assert nat.PlanKD((30, 20), (8, 4)).launch_count() == 1      # fused form for small windows
    assert nat.PlanKD((300, 200), (32, 16)).launch_count() == 2



# ------------------------------------------------------------------ streaming (swdftstream.h)

@pytest.mark.parametrize("args,status", [
    ((0, 4, 4, 0, 0, 1), -1),      # empty row
    ((16, 3, 4, 0, 0, 1), -2),     # not a power of two
    ((16, 4, 32, 0, 0, 1), -3),    # window wider than the row
    ((300, 128, 4, 0, 0, 1), -4),  # beyond the 64-point axis
    ((16, 4, 4, 5, 0, 1), -1),     # bad dtype
    ((16, 4, 4, 0, 9, 1), -1),     # bad normalisation
    ((16, 4, 4, 0, 0, 0), -1),     # no rows per push
])
def test_stream_validation(nat, args, status):
    st, h = nat.raw_stream(*args)
    assert st == status
    assert h is None


def test_stream_state_and_push_bookkeeping(nat):
    s = nat.StreamPlan(40, 8, 4, max_rows=5)
    # n1 <= 32, max_rows <= 4 n0: 2(n0-1) + max_rows kept input rows of N1 float32
    assert s.state_size() == (14 + 5) * 40 * 4
    # otherwise: n0/2 look-back rows + 2(n0-1) + max_rows kept z rows of P1*n1 complex64
    assert nat.StreamPlan(70, 8, 64, max_rows=5).state_size() == (4 + 14 + 5) * 7 * 64 * 8
    assert nat.StreamPlan(40, 8, 4, max_rows=33).state_size() == (4 + 14 + 33) * 37 * 4 * 8
    # pushes of zero rows enqueue nothing and need no pointers
    assert s.push(0, 0, 0, 0, 0) == (0, 0)
    assert s.rows_seen() == 0
    with pytest.raises(nat.SwdftError):
        s.push(0, 6, 0, 0, 0)      # more rows than max_rows
    with pytest.raises(nat.SwdftError):
        s.push(0, 2, 20, 0, 0)     # row stride shorter than a row


def test_persistent_batch_launches_one_kernel_per_window_class(nat):
    """A persistent plan runs one kernel per window shape (n0, n1), pipelined or fused,
    whatever the number of arrays: repeating arrays adds no launch, and the 256-image uneven
    batch needs one per distinct window shape."""
    import workloads
    one = [shp(256, 256, 4, 4), shp(512, 128, 32, 32), shp(128, 1024, 64, 16)]
    base = nat.Plan(one, flags=nat.FLAG_PERSISTENT).launch_count()
    assert base == 3
    for k in (2, 7, 40):
        assert nat.Plan(one * k, flags=nat.FLAG_PERSISTENT).launch_count() == base
    # per-array plans launch once or twice per array instead
    assert nat.Plan(one * 7).launch_count() >= 7 * 3
    _, sides, widx = workloads.uneven_batch_shapes()
    shapes = [shp(int(sides[i, 0]), int(sides[i, 1]), *workloads.UNEVEN_WINDOWS[int(widx[i])])
              for i in range(len(widx))]
    windows = {workloads.UNEVEN_WINDOWS[int(w)] for w in widx}
    n_pers = nat.Plan(shapes, flags=nat.FLAG_PERSISTENT).launch_count()
    assert n_pers == len(windows) == 6
    assert nat.Plan(shapes).launch_count() >= len(shapes)


def test_forms_of_a_persistent_plan(nat):
    """swdft2d_get_form: in a persistent plan, two-pass windows run pipelined, small windows
    (n0 n1 <= 64, n1 < 64) in fused groups, tensor-core arrays on their own; without the flag
    every array runs on its own."""
    shapes = [shp(100, 90, 32, 32), shp(20, 20, 4, 4), shp(70, 130, 1, 64), shp(64, 64, 16, 4)]
    p = nat.Plan(shapes, flags=nat.FLAG_PERSISTENT)
    assert [p.form(i) for i in range(4)] == [("tree", "pipelined"), ("tree", "fused_group"),
                                            ("tree", "pipelined"), ("tree", "fused_group")]
    q = nat.Plan(shapes)
    assert [q.form(i)[1] for i in range(4)] == ["per_array"] * 4
    tc = nat.Plan([shp(100, 90, 32, 32), shp(70, 130, 16, 64)], algo="tc_bf16x3",
                  flags=nat.FLAG_PERSISTENT)
    assert [tc.form(i) for i in range(2)] == [("tc_bf16x3", "per_array")] * 2
    assert tc.launch_count() == 4
    with pytest.raises(nat.SwdftError):
        p.form(4)
    mixed = nat.Plan([shp(100, 90, 27, 27), shp(100, 90, 12, 16), shp(100, 90, 32, 32)], flags=nat.FLAG_PERSISTENT)
    assert [mixed.form(i)[1] for i in range(3)] == ["per_array", "per_array", "pipelined"]
    assert mixed.launch_count() == 2 + 2 + 1


def test_persistent_workspace_holds_z_regions_and_the_pipeline_counters(nat):
    """A persistent plan's workspace: every array's own region (its z, or its adjoint's gz and
    side rows), then one block of counters for the pipelined kernels -- 64 words, then a flag
    per row tile (row block of z rows x row chunk of window columns) of every array (the
    autotuner may move any array into a pipelined kernel), 256-byte aligned.  So a batch takes
    its arrays' single-array workspaces less all but one counter block."""
    r = lambda b: (b + 255) // 256 * 256
    A, B, C = shp(100, 90, 32, 32), shp(20, 20, 4, 4), shp(70, 130, 16, 64)
    ws = lambda shapes: nat.Plan(shapes, flags=nat.FLAG_PERSISTENT).workspace_size()
    # row tiles: ceil(z rows / (128 >> B)) x ceil(P1 / chunk), B = 3 for n1 >= 8 (m1 for
    # n1 < 8), chunk = max(n1 / 2, P1 over ~64K threads)
    f = {"A": -(-(69 + 31) // 16) * -(-59 // 16), "B": -(-(17 + 3) // 32) * -(-17 // 2),
         "C": -(-(55 + 15) // 16) * -(-67 // 32)}
    shape = {"A": A, "B": B, "C": C}
    cnt = lambda flags: r(4 * (64 + flags))
    region = {x: ws([shape[x]]) - cnt(f[x]) for x in "ABC"}
    for batch in ("ABC", "AA", "BB", "A" * 10 + "C" * 7 + "B" * 3):
        assert ws([shape[x] for x in batch]) == sum(region[x] for x in batch) + cnt(sum(f[x] for x in batch))
    assert cnt(10 * f["A"] + 7 * f["C"] + 3 * f["B"]) == 2048  # 64 + 412 words, 256-byte aligned


def test_injected_allocation_failures(nat):
    """swdft2d_inject_alloc_failure: with no allocation left every plan, kD plan and stream
    creation fails with SWDFT_ERR_OOM and leaves no handle; with one left the first creation
    succeeds and the next fails; after < 0 restores normal behaviour."""
    try:
        nat.inject_alloc_failure(0)
        st, h = nat.raw_plan([shp(16, 16, 4, 4)], 0, 0, 1, 0)
        assert st == -5 and h is None
        with pytest.raises(nat.SwdftError) as e:
            nat.PlanKD((8, 8, 8), (2, 2, 2))
        assert e.value.status == -5
        st, h = nat.raw_stream(16, 4, 4, 0, 0, 1)
        assert st == -5 and h is None
        nat.inject_alloc_failure(1)
        p = nat.Plan([shp(16, 16, 4, 4)])
        with pytest.raises(nat.SwdftError) as e:
            nat.Plan([shp(16, 16, 4, 4)])
        assert e.value.status == -5
        assert p.output_shape(0) == (13, 13, 4, 4)
        # invalid arguments are still reported as such, before any allocation
        st, _ = nat.raw_plan([shp(16, 16, 5, 4)], 0, 0, 1, 0)
        assert st == -2
    finally:
        nat.inject_alloc_failure(-1)
    assert nat.Plan([shp(16, 16, 4, 4)]).output_shape(0) == (13, 13, 4, 4)
    assert nat.StreamPlan(16, 4, 4).state_size() > 0


def test_selftest_wait_timeout_checks_its_argument_first(nat):
    for polls in (0, -3, 4097):
        with pytest.raises(nat.SwdftError) as e:
            nat.selftest_wait_timeout(polls)
        assert e.value.status == -1


def _tune_line(gpu, N0, N1, n0, n1, algo=1, auto=0, fused=0, row_B=2, row_chunk=0, col_B=2, col_chunk=0,
               col_groups=1, dtype=0, ld=None, q_begin=0, q_end=None):
    """One tuning-cache record in the layout swdft2d_autotune writes."""
    rec = {"gpu": gpu, "N0": N0, "N1": N1, "ld": N1 if ld is None else ld, "n0": n0, "n1": n1,
           "dtype": dtype, "q_begin": q_begin, "q_end": N0 - n0 + 1 if q_end is None else q_end,
           "auto": auto, "algo": algo, "fused": fused, "row_B": row_B, "row_chunk": row_chunk,
           "col_B": col_B, "col_chunk": col_chunk, "col_groups": col_groups, "ms": 0.125}
    return json.dumps(rec) + "\n"


def test_load_tuning_applies_records_of_the_named_gpu(nat, tmp_path):
    """swdft2d_load_tuning on the host: the last applicable record for the named GPU sets the
    array's choice (here the fused form: one launch instead of two, and the tensor-core form
    for an AUTO plan); other GPUs, other arrays, choices the plan cannot run and lines in
    another layout are ignored."""
    cache = tmp_path / "tune.jsonl"
    assert nat.Plan([shp(300, 300, 16, 16)]).load_tuning(str(tmp_path / "missing.jsonl"), "G") == 0
    cache.write_text(
        "not a record\n" +
        _tune_line("Other GPU", 300, 300, 16, 16, fused=1) +
        _tune_line("Test GPU", 300, 300, 16, 16, fused=0) +
        _tune_line("Test GPU", 300, 300, 16, 16, fused=1, row_chunk=64, col_chunk=32) +   # last wins
        _tune_line("Test GPU", 300, 300, 16, 16, fused=1, row_B=7) +                      # invalid split
        _tune_line("Test GPU", 300, 301, 16, 16, fused=1) +                               # another array
        _tune_line("Test GPU", 300, 300, 16, 16, algo=2, auto=1))                         # AUTO plans only
    p = nat.Plan([shp(300, 300, 16, 16)])
    assert p.launch_count() == 2
    assert p.load_tuning(str(cache), "Other GPU") == 1 and p.launch_count() == 1
    p = nat.Plan([shp(300, 300, 16, 16)])
    assert p.load_tuning(str(cache), "Another GPU") == 0 and p.launch_count() == 2
    two = nat.Plan([shp(300, 300, 16, 16), shp(64, 64, 8, 8)])
    assert two.load_tuning(str(cache), "Test GPU") == 1
    assert two.launch_count() == 1 + 1  # the first fused now; the second (8x8) was fused already
    auto = nat.Plan([shp(300, 300, 16, 16)], algo="auto")
    assert auto.algo() == "tree"
    assert auto.load_tuning(str(cache), "Test GPU") == 1 and auto.algo() == "tc_bf16x3"
    band = nat.Plan([shp(300, 300, 16, 16, row_begin=10, row_end=50)])
    assert band.load_tuning(str(cache), "Test GPU") == 0
    import torch
    if not torch.cuda.is_available():  # no device to take the GPU name from
        with pytest.raises(nat.SwdftError) as e:
            nat.Plan([shp(300, 300, 16, 16)]).load_tuning(str(cache))
        assert e.value.status == -6


def test_load_tuning_rejects_chunks_beyond_the_grid_limit(nat, tmp_path):
    """A record whose row or column chunks would cut this array's pass into more than 65535
    pieces (the grid's y limit) is not applied: the array keeps its default choice, and the
    record that fits is applied."""
    cache = tmp_path / "tune.jsonl"
    N0, N1 = 70000, 40
    cache.write_text(
        _tune_line("G", N0, N1, 2, 2, fused=0, col_chunk=1, col_B=1, row_B=1) +      # 69999 chunks
        _tune_line("G", 300, 70000, 2, 2, fused=0, row_chunk=1, col_B=1, row_B=1))   # 69999 chunks
    tall = nat.Plan([shp(N0, N1, 2, 2)])
    assert tall.load_tuning(str(cache), "G") == 0
    wide = nat.Plan([shp(300, 70000, 2, 2)])
    assert wide.load_tuning(str(cache), "G") == 0
    cache.write_text(_tune_line("G", N0, N1, 2, 2, fused=0, col_chunk=2, col_B=1, row_B=1))
    assert nat.Plan([shp(N0, N1, 2, 2)]).load_tuning(str(cache), "G") == 1


def test_fused_form_covers_n1_64_up_to_n0_32(nat):
    """The fused form (one launch) is built for n1 <= 32 and for n1 = 64 with n0 <= 32: a plan
    asked for it on 16x64 or 1x64 windows runs one kernel; on 64x64 windows it keeps two passes."""
    for (n0, n1), want in (((16, 64), 1), ((1, 64), 1), ((32, 64), 1), ((64, 64), 2), ((64, 32), 1)):
        p = nat.Plan([shp(200, 200, n0, n1)])
        p.set_tree_config(0, 2, 0, 2, 0, 1, 1)
        assert p.launch_count() == want, (n0, n1)
    # 1024x2048 complex with 16x64 windows: z would be 1 GB, so the default is the fused form
    assert nat.Plan([shp(1024, 2048, 16, 64, dtype=nat.C64)]).launch_count() == 1
