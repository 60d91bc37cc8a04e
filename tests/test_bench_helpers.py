"""Host helpers of bench.py that decide what the benchmark line reports (no GPU): the solve kernel's code hash
ignores comments and whitespace but not code, so a committed DRAM-traffic record stays valid across comment
edits and lapses with any code change; a traffic record is used only for the workload it was taken on; and
the algorithmic byte model adds the per-step, per-round and per-iteration terms its docstring states."""
import bench


def test_code_tokens_ignore_comments_and_whitespace():
    a = "int f(int x) {  // add one\n  return x + 1; /* done\n   twice */ }\n"
    b = "int f(int x)\n{\n return x + 1;\n}"
    assert bench.code_tokens(a) == bench.code_tokens(b)
    assert bench.code_tokens(a) != bench.code_tokens(a.replace("x + 1", "x + 2"))


def test_source_hash_tracks_code_not_comments():
    files = {"kernels_solve.cu": "__global__ void k() { int a = 1; }\n", "internal.h": "struct S { int n; };\n"}
    h0 = bench.solve_source_hash(read=files.__getitem__)
    commented = dict(files, **{"kernels_solve.cu": "// note\n__global__ void k() {\n  int a = 1;  /* x */\n}\n"})
    assert bench.solve_source_hash(read=commented.__getitem__) == h0
    changed = dict(files, **{"internal.h": "struct S { long n; };\n"})
    assert bench.solve_source_hash(read=changed.__getitem__) != h0


def test_traffic_record_only_for_its_workload():
    assert bench.measured_traffic("no-such-workload") == (None, None)
    traffic, algo = bench.measured_traffic("batch256")
    if traffic is not None:   # the committed record was taken on the current solve-kernel source
        assert algo is not None and 0.5 < traffic / algo < 2.0


def test_algorithmic_bytes_terms():
    info = {"n_verts": 1000, "nnz": 19000, "n_slots": 6000, "vcycle_bytes": 5e5}
    stats = {"total_refine_rounds": 3, "total_pcg_iterations": 20}
    per_step = 16 * 6000 + (213 + 240) * 1000
    per_round = 12 * 19000 + 240 * 1000 + 5e5
    per_iter = 8 * 19000 + 192 * 1000 + 5e5
    assert bench.algorithmic_bytes(info, stats, 2) == 2 * per_step + 3 * per_round + 20 * per_iter
    # exact backward Euler, three chord solves in the step: the slots twice more, and per later solve the
    # product (A - M) v_k, its right-hand side and the hand-off to the next iterate
    extra = bench.algorithmic_bytes(info, dict(stats, nl_iterations=3), 1) - bench.algorithmic_bytes(info, stats, 1)
    assert extra == 2 * 16 * 6000 + 2 * (12 * 19000 + (32 + 109 + 104) * 1000)


def test_force_phase_bytes():
    base = {"n_verts": 1000, "nnz": 19000, "n_slots": 6000, "vcycle_bytes": 0, "n_tris": 1900, "n_stencils": 2800}
    stats = {"total_refine_rounds": 0, "total_pcg_iterations": 0}
    tri = bench.algorithmic_bytes(dict(base, model="SP"), stats, 1) - bench.algorithmic_bytes(base, stats, 1)
    assert tri == 244 * 1900 + 24 * 1000
    edge = bench.algorithmic_bytes(dict(base, model="ES"), stats, 1) - bench.algorithmic_bytes(base, stats, 1)
    assert edge == 88 * 1900 + 89 * 2800 + 24 * 1000
    # every chord solve of an exact backward-Euler step evaluates the forces again
    two = bench.algorithmic_bytes(dict(base, model="SP"), dict(stats, nl_iterations=2), 1)
    one = bench.algorithmic_bytes(base, dict(stats, nl_iterations=2), 1)
    assert two - one == 2 * (244 * 1900 + 24 * 1000)


def test_scaled_traffic_uses_the_capture_ratio_on_the_current_source():
    rec = {"source_sha1": bench.solve_source_hash(), "workload": "batch128", "traffic_bytes_per_launch": "4.4e9",
           "algorithmic_bytes_of_captured_launch": "4.0e9"}
    est, ratio, wl = bench.scaled_traffic(8.0e9, record=rec)
    assert wl == "batch128" and abs(ratio - 1.1) < 1e-12 and abs(est - 8.8e9) < 1.0
    assert bench.measured_traffic("batch256", record=rec) == (None, None)
    stale = dict(rec, source_sha1="0" * 40)
    assert bench.scaled_traffic(8.0e9, record=stale) == (None, None, None)


def test_bytes_without_vcycle_drop_only_the_cycle_terms():
    info = {"n_verts": 1000, "nnz": 19000, "n_slots": 6000, "vcycle_bytes": 5e5}
    stats = {"total_refine_rounds": 3, "total_pcg_iterations": 20}
    full = bench.algorithmic_bytes(info, stats, 2)
    assert full - bench.algorithmic_bytes_without_vcycle(info, stats, 2) == (3 + 20) * 5e5
