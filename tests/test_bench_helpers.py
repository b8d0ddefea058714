"""Host logic of bench.py (no GPU): the kernel-code digest that keys the DRAM
traffic table ignores comments but not code, the committed table parses and
is reported only for the captured kernel code, and the launch-shape tags."""
import os

import bench


def test_code_digest_ignores_comments_only():
    a = "int f(int x) { return x + 1; }  // one\n/* block */\n"
    b = "// other\nint f(int x) { return x + 1; }\n\n/* a\n longer block */"
    c = "int f(int x) { return x + 2; }\n"
    assert bench._code_only(a) == bench._code_only(b)
    assert bench._code_only(a) != bench._code_only(c)


def test_traffic_table_matches_current_kernels():
    rows = [ln for ln in open(bench.TRAFFIC_FILE).read().splitlines()
            if ln.strip() and not ln.startswith("#")]
    assert rows
    digest = bench.sources_digest()
    for ln in rows:
        f = [x.strip() for x in ln.split("|")]
        assert len(f) == 5 and int(f[2]) >= 0 and int(f[3]) >= 0
        got = bench.measured_traffic(f[0], f[1])
        # reported while the kernel code is the captured one, null after a change
        assert got == (int(f[2]) + int(f[3]) if f[4] == digest else None)
    assert bench.measured_traffic("k_neighbours_direct", "no-such-workload") is None


def test_tuning_tag():
    assert bench.tuning_tag({"mode": 2, "stencil": 1, "block": 128, "lanes": 2}) == "m2-s1-b128-l2"
    assert bench.tuning_tag({"mode": 1, "stencil": 2, "block": 256, "tile_w": 16,
                             "tile_h": 4}) == "m1-s2-b256-t16x4"
