"""The committed trained picker (data/picker_config4.npz) and its report,
checked on the CPU with the fp64 oracle network: its bf16 working copy is the
fp32 master rounded to nearest even, its feature normalisation is valid; on
the committed held-out set (features and the measured chain time of every
schedule on 512 held-out tiles) the oracle network's picks reproduce the
report's picks and its gain over the plain schedule, which is above 1 on a
set where every class is the best one for some tiles; and the robustness
study's confidence fall-back keeps the picks no slower than the plain
schedule under every feature noise it tried, while without the fall-back
the noise costs time."""
import json
import os

import numpy as np

from oracle import mlp as OM

DATA = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1405_7958_gb300", "data")
PLAIN = 3     # the fall-back class: the times' column of the plain schedule (raster, 12 iterations)


def _load():
    return np.load(os.path.join(DATA, "picker_config4.npz"))


def _report():
    with open(os.path.join(DATA, "picker_config4_report.json")) as fh:
        return json.load(fh)


def test_picker_parameters_are_consistent():
    z = _load()
    assert z["master"].shape == (OM.NPARAM,) and z["wb"].shape == (OM.NPARAM,)
    assert z["m"].shape == (OM.NPARAM,) and z["v"].shape == (OM.NPARAM,)
    assert z["norm"].shape == (2 * OM.NIN,) and (z["norm"][OM.NIN:] > 0).all()
    assert int(z["step_count"]) > 0 and np.isfinite(z["master"]).all()
    u = z["master"].view(np.uint32).astype(np.uint64)
    rne = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint16)
    assert np.array_equal(rne, z["wb"].astype(np.uint16))


def test_oracle_network_reproduces_the_held_out_report():
    z, r = _load(), _report()
    ev = np.load(os.path.join(DATA, "picker_config4_report_eval_set.npz"))
    feats, times = ev["feats"].astype(np.float64), ev["times"]
    p = OM.bf16_bits_to_f64(z["wb"])
    logits = OM.forward(p, z["norm"].astype(np.float64), feats)[3]
    pick = logits.argmax(axis=1)
    counts = [int((pick == k).sum()) for k in range(3)]
    want = list(r["eval"]["pick_counts"].values())[:3]
    # fp64 here, fp32 on the GPU: only near-ties may differ
    assert sum(abs(a - b) for a, b in zip(counts, want)) <= 0.02 * len(pick)
    best = times[:, :PLAIN].argmin(axis=1)
    assert all((best == k).sum() >= 0.01 * len(best) for k in range(3))   # every class is sometimes the best
    chosen = times[np.arange(len(times)), pick].sum()
    gain = times[:, PLAIN].sum() / chosen
    assert abs(gain - r["eval"]["gain_vs_plain"]) < 0.003
    assert gain > 1.0                                                    # faster than the plain schedule
    assert chosen >= times[:, :PLAIN].min(axis=1).sum()


def test_report_is_consistent():
    r = _report()
    for part in ("train", "eval"):
        ev = r[part]
        assert sum(ev["pick_counts"].values()) == ev["tiles"] == sum(ev["best_counts"].values())
        assert ev["time_best_ms"] <= ev["time_learned_ms"] <= ev["time_worst_ms"]
        assert ev["time_best_ms"] <= ev["time_plain_ms"] <= ev["time_worst_ms"]
        assert 0.0 <= ev["accuracy"] <= 1.0 and ev["regret_mean_ms"] >= 0.0
    assert [s["max_local"] for s in r["schedules"]] == [4, 12, 24] and r["plain_class"] == PLAIN
    assert r["plain_schedule"] == {"variant": 1, "max_local": 12}


def test_fall_back_bounds_the_loss_under_estimate_errors():
    """The paper's PATS evaluation perturbs the estimates its scheduler uses;
    here Gaussian noise on the picker's features: with the confidence
    fall-back at 0.95 no draw at any noise level is slower than the plain
    schedule, and without it noise does cost time (the picks drift towards
    slower schedules; under heavy noise the network extrapolates with more
    confidence, so fewer picks fall back)."""
    rows = [x for x in _report()["robustness_eval"] if "sigma" in x]
    bounds = [x for x in _report()["robustness_eval"] if "bounds" in x][0]["bounds"]
    fb = {x["sigma"]: x for x in rows if x["min_prob"] == 0.95}
    assert all(x["time_vs_plain_max"] <= 1.0 for x in fb.values())
    assert all(bounds["best_vs_plain"] <= x["time_vs_plain"] <= bounds["worst_vs_plain"] for x in rows)
    nofb = [x for x in rows if x["min_prob"] == 0.0]
    assert all(x["fell_back"] == 0.0 for x in nofb)
    sig = sorted(fb)
    nofb = {x["sigma"]: x for x in nofb}
    assert nofb[sig[-1]]["time_vs_plain"] >= nofb[sig[0]]["time_vs_plain"]     # noise costs
