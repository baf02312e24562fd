"""The autotuner's host logic (no device): how a point of its search space becomes
context options, and the shape of that space."""
from paper_2009_04061_gb300 import autotune


def test_options_of_a_point():
    o = autotune._options({"hist_variant": 0, "hist_chunk": 16, "search_slots_per_sm": 12,
                           "small_search_nodes": 32, "small_search_warps": 20}, sms=152)
    assert o == {"hist_variant": 0, "hist_chunk": 16, "search_slots": 12 * 152,
                 "small_search_nodes": 32, "small_search_warps": 20}
    # 0 warps per SM for the global-memory tier means the library default: no option
    assert "search_slots" not in autotune._options({"search_slots_per_sm": 0}, sms=152)
    # the chunk schedules only the window kernel
    assert "hist_chunk" not in autotune._options({"hist_variant": 2, "hist_chunk": 16}, sms=152)


def test_search_space_starts_at_the_library_defaults():
    names = [n for n, _ in autotune.DIMENSIONS]
    assert len(names) == len(set(names))
    first = {n: v[0] for n, v in autotune.DIMENSIONS}
    assert first["hist_variant"] == 0 and first["hist_chunk"] == 24 and first["reach_schedule"] == 0
    assert first["small_search_nodes"] == 64 and first["small_search_warps"] == 24
    assert first["search_slots_per_sm"] == 0
    assert all(n in autotune.PHASE for n in names)
    for n, values in autotune.DIMENSIONS:
        if n == "small_search_warps":
            assert all(v % 4 == 0 and 0 < v <= 32 for v in values)
