"""Host-side helpers of bench.py on the CPU: the fixed-error comparison of the surrogate
and table paths, the code-only hash that ties an ncu summary to the kernel sources,
and the multi-GPU camera split.  No GPU is used."""
import numpy as np
import pytest

import bench
from paper_2512_01283_gb300 import multigpu as MG


def _maps(rng, truth, sigma, bias=0.0):
    return truth * (1.0 + bias) + sigma * rng.standard_normal(truth.shape)


def test_fixed_error_recovers_spread_and_bias():
    """Synthetic maps with known Monte-Carlo spread and systematic difference: the
    estimates come back, and the packets to a target error follow eps^2 = b^2 +
    sigma^2 N0 / N."""
    rng = np.random.default_rng(3)
    truth = rng.random((8, 4, 96, 96)) + 1.0
    rms = float(np.sqrt(np.mean(truth[:, 0] ** 2)))
    t1, t2 = _maps(rng, truth, 0.05), _maps(rng, truth, 0.05)
    s1, s2 = _maps(rng, truth, 0.08, 0.01), _maps(rng, truth, 0.08, 0.01)
    fe = bench.fixed_error(t1, t2, s1, s2, 1e8, 1.5, 12.0)
    I = fe["I"]
    assert I["sigma_table"] == pytest.approx(0.05 / rms, rel=0.03)
    assert I["sigma_surrogate"] == pytest.approx(0.08 / rms, rel=0.03)
    assert I["bias_surrogate"] == pytest.approx(0.01, abs=0.002)
    for row in I["targets"]:
        eps = row["eps"]
        assert row["table_packets"] == pytest.approx(1e8 * I["sigma_table"] ** 2 / eps ** 2)
        assert row["table_s"] == pytest.approx(row["table_packets"] / 1e8 * 1.5)
        if eps > I["bias_surrogate"]:
            n = 1e8 * I["sigma_surrogate"] ** 2 / (eps ** 2 - I["bias_surrogate"] ** 2)
            assert row["surrogate_packets"] == pytest.approx(n)
            assert row["table_over_surrogate_time"] == pytest.approx(row["table_s"] / row["surrogate_s"])


def test_fixed_error_without_bias_and_out_of_reach():
    rng = np.random.default_rng(4)
    truth = rng.random((4, 4, 64, 64)) + 1.0
    t1, t2 = _maps(rng, truth, 0.05), _maps(rng, truth, 0.05)
    same = bench.fixed_error(t1, t2, t2, t1, 1e8, 1.0, 1.0)  # the surrogate is the table path
    assert same["I"]["bias_surrogate"] == 0.0
    far = bench.fixed_error(t1, t2, t1 * 1.2, t2 * 1.2, 1e8, 1.0, 1.0)  # 20 % off
    assert far["I"]["bias_surrogate"] > 0.15
    row = far["I"]["targets"][0]
    assert row["surrogate_packets"] is None and row["surrogate_s"] is None


def test_code_only_drops_comments_and_blank_space():
    a = "int a = 1;  // one\n/* block\n comment */ float b;\n"
    b = "int a = 1;\n\n   float b; // other words\n"
    assert bench.code_only(a) == bench.code_only(b) == "int a = 1; float b;"
    assert bench.code_only("int a = 2;") != bench.code_only(a)


def test_kernel_hash_ignores_comments_only():
    src = {f: "__global__ void k() { int x = 1; }\n" for f in bench.KERNEL_SOURCES}
    h0 = bench.kernel_source_sha(lambda f: src[f])
    commented = {f: "// header\n" + t + "/* end */\n" for f, t in src.items()}
    assert bench.kernel_source_sha(lambda f: commented[f]) == h0
    changed = dict(src)
    changed[bench.KERNEL_SOURCES[0]] = "__global__ void k() { int x = 2; }\n"
    assert bench.kernel_source_sha(lambda f: changed[f]) != h0


def test_committed_summary_matches_the_kernel_sources():
    """The committed ncu summary of the table rounds belongs to the kernel code as it
    stands, so bench.py reports its traffic and issue figures."""
    f = bench.profiled_fields()
    assert f, "profiles/rounds_disk192.md is stale or missing"
    assert float(f["transport_traffic_bytes_per_unit"]) > 0
    assert bench.profiled_traffic("tally", 10.0) == pytest.approx(10.0 * float(f["tally_traffic_bytes_per_unit"]))
    issue = bench.profiled_issue("transport")
    assert 0.0 < issue["issue_active"] <= 1.0 and 1.0 <= issue["threads_per_warp_instruction"] <= 32.0


def test_camera_split_for_every_world_size():
    for world in range(1, 9):
        seen = [k for r in range(world) for k in MG.rank_cameras(8, r, world)]
        assert sorted(seen) == list(range(8))
