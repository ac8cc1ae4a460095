"""The autotuner's search (coordinate descent over (k, block bytes), the
base-case size and alpha), on the CPU with a synthetic cost function."""
from paper_2009_13569_gb300 import autotune


def test_search_finds_the_separable_minimum():
    # cost = f(kb) + g(base) + h(alpha): coordinate descent reaches the optimum
    def cost(p):
        kb = {(256, 512): 3.0, (128, 1024): 1.0, (64, 2048): 2.0, (128, 512): 2.5,
              (64, 1024): 1.5, (64, 512): 4.0}[(p["k"], p["block_bytes"])]
        base = abs(p["base_case"] - autotune.base_cap("u64") // 2) / 1000.0
        alpha = {0.2: 0.3, 0.5: 0.1, 1.0: 0.2}[p["alpha_scale"]]
        return kb + base + alpha

    best, table = autotune.search(cost, "u64")
    assert (best["k"], best["block_bytes"]) == (128, 1024)
    assert best["base_case"] == autotune.base_cap("u64") // 2
    assert best["alpha_scale"] == 0.5
    # every candidate timed once, the starting point not twice
    keys = [tuple(sorted(p.items())) for p, _ in table]
    assert len(keys) == len(set(keys)) == len(autotune.KB_PAIRS) + 2 + 2


def test_search_skips_rejected_candidates():
    def cost(p):
        if p["k"] == 256:
            return None  # e.g. refused by the library
        return 1.0 if p["k"] == 64 else 2.0

    best, table = autotune.search(cost, "u32")
    assert best["k"] == 64
    assert any(t is None for _, t in table)


def test_every_kb_pair_fits_one_classification_cta():
    # k * block bytes at most 128 KiB, blocks at most 2 KiB, as the library accepts
    for k, bb in autotune.KB_PAIRS:
        assert k * bb <= 128 * 1024 and bb <= 2048
        for dtype in ("u32", "u64", "pair", "rec100", "quartet"):
            from paper_2009_13569_gb300 import ipsgpu
            assert ipsgpu.scratch_bytes(dtype, k=k, block_bytes=bb) > 0, (dtype, k, bb)


def test_base_cap_matches_the_library_limit():
    assert autotune.base_cap("u64") == 184 * 1024 // 8
    assert autotune.base_cap("rec100") == 184 * 1024 // 100


def test_cache_file_stores_and_reuses(tmp_path):
    path = str(tmp_path / "tune.json")
    calls = []

    def tune():
        calls.append(1)
        return {"k": 128, "block_bytes": 1024, "alpha_scale": 0.5, "base_case": 100}, [("t", 1.0)]

    best, table = autotune.cached(path, "array:u64:n=1024", tune)
    assert len(calls) == 1 and table
    again, table2 = autotune.cached(path, "array:u64:n=1024", tune)
    assert again == best and table2 == [] and len(calls) == 1  # hit: nothing timed
    other, _ = autotune.cached(path, "array:u64:n=2048", tune)
    assert len(calls) == 2  # another workload shape is tuned again
    assert autotune.cached(None, "x", tune)[1]  # no cache file: always tuned


def test_segmented_signature_is_coarse():
    a = autotune.segmented_signature([0, 1, 3, 1000, 1023])
    b = autotune.segmented_signature([0, 1, 2, 600, 1020])
    assert a.startswith("arrays=5,")
    # same histogram of log2 lengths, different totals: different keys
    assert a.split("log2hist=")[1] == b.split("log2hist=")[1] and a != b
