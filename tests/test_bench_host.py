"""Host checks of the benchmark's bookkeeping: the per-launch DRAM counters under
profiles/ parse into known workloads, kernel kinds and tile-menu entries, and
the kernel-source hashes they are keyed by are computed over the regions the
benchmark documents."""
import re

import bench

MENU_SIZE = 16   # entries of the stencil tile menu (hv_tile_menu_size)


def test_dram_counters_parse():
    table = bench.dram_traffic()
    assert table, "profiles/dram_traffic.txt holds no entries"
    for (workload, kind, tile), (h, nbytes) in table.items():
        assert workload in ("paper", "batched", "batched-resident", "misfits"), workload
        assert kind in ("fwd", "advance", "adj"), kind
        assert re.fullmatch(r"[0-9a-f]{16}", h), h
        assert nbytes > 0
        assert (tile == 0) if workload.endswith("resident") else (0 <= tile < MENU_SIZE), (workload, tile)


def test_source_hashes_cover_nested_regions():
    tiled, resident = bench.csrc_hash(False), bench.csrc_hash(True)
    assert re.fullmatch(r"[0-9a-f]{16}", tiled) and re.fullmatch(r"[0-9a-f]{16}", resident)
    # the resident region extends the tiled one, so the two hashes differ
    assert tiled != resident
