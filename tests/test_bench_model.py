"""Host-side checks of bench.py's roofline accounting (no GPU): per-launch work
and time must not depend on how many timed builds the totals cover."""
import bench
from paper_2010_11497_gb300 import synth

W10 = synth.WORKLOADS["ml10m_like"]
STATS = {"greedy_visits": 716_434_200, "greedy_computed": 796_038, "greedy_users": 176_135,
         "greedy_evaluated": 219_512_800, "item_visits_brute": 0,
         "item_visits_greedy": 457_714_162, "brute_gram_elems": 61_725_056,
         "brute_rows": 354_257}
PER_BUILD_MS = {"validate": 0.08, "hash_minhash_level0": 0.16, "split": 0.38, "gram": 1.38,
                "brute_rows": 0.75, "greedy_init": 1.01, "greedy_rounds": 3.13, "merge": 0.27}
PEAKS = {"hbm_gbs": 6780.7, "sm_max_mhz": 2070.0}


def _rows(steps):
    ms = {k: v * steps for k, v in PER_BUILD_MS.items()}
    calls = {k: steps for k in ms}
    return bench.roofline(ms, calls, STATS, W10, 10_034_432, PEAKS, "measured", 1, steps)


def test_per_launch_figures_do_not_depend_on_steps():
    rf1, rows1 = _rows(1)
    rf5, rows5 = _rows(5)
    assert rf1["kernel"] == rf5["kernel"] == "k_greedy_round"
    assert abs(rf1["frac"] - rf5["frac"]) < 1e-12
    by1 = {r["phase"]: r for r in rows1}
    by5 = {r["phase"]: r for r in rows5}
    for ph in ("gram", "brute_rows", "merge", "hash_minhash_level0"):
        assert abs(by1[ph]["frac"] - by5[ph]["frac"]) < 1e-12, ph
        assert abs(by1[ph]["ms_per_launch"] - PER_BUILD_MS[ph]) < 1e-12, ph


def test_models_match_hand_computation():
    _, rows = _rows(3)
    by = {r["phase"]: r for r in rows}
    alu_peak = 152 * 128 * 2070e6 / 1e12
    # greedy: 12 lane-ops per examined entry, one launch per round
    ach = STATS["greedy_visits"] / 10 * 12 / (PER_BUILD_MS["greedy_rounds"] / 10 * 1e-3) / 1e12
    assert abs(by["greedy_rounds"]["achieved"] - ach) < 1e-9 * ach
    assert abs(by["greedy_rounds"]["peak"] - alu_peak) < 1e-9
    # count matrices, W = 1 (bit-sliced counts): table load, item unpack, 15
    # full adders of 2 logic ops per 16 items, the weight-16 carry through at
    # most 12 planes: 1 + 1 + 30/16 + 24/16 = 5.375 lane-ops per item visit
    ach = STATS["item_visits_greedy"] * 5.375 / (PER_BUILD_MS["gram"] * 1e-3) / 1e12
    assert abs(by["gram"]["achieved"] - ach) < 1e-9 * ach
    # merge: t rows of k (id, inter, union) per user read, one row written, slot map
    n, t, k = W10.n_users, W10.t, W10.k
    byts = 4 * t * n + 12 * t * n * k + 12 * n * k
    assert abs(by["merge"]["achieved"] - byts / (PER_BUILD_MS["merge"] * 1e-3) / 1e9) < 1e-6
    # shares add up to one and the dominant phase comes first
    assert abs(sum(r["share"] for r in rows) - 1.0) < 1e-9
    assert rows[0]["phase"] == "greedy_rounds"


def test_two_word_table_model():
    # two-word tables keep 4-bit SWAR counters: 1 + W + 12 W + 48 W / 12 = 35
    # lane-ops per item visit at W = 2
    ms = dict(PER_BUILD_MS)
    calls = {k: 1 for k in ms}
    _, rows = bench.roofline(ms, calls, STATS, W10, 10_034_432, PEAKS, "measured", 2, 1)
    by = {r["phase"]: r for r in rows}
    ach = STATS["item_visits_greedy"] * 35 / (PER_BUILD_MS["gram"] * 1e-3) / 1e12
    assert abs(by["gram"]["achieved"] - ach) < 1e-9 * ach
    assert by["gram"]["kernel"] == "k_gram<2>"
