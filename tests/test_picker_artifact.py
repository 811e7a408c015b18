"""The committed trained picker (data/picker_config4.npz), checked on the CPU
with the fp64 oracle network and oracle features: its bf16 working copy is
the fp32 master rounded to nearest even, its feature normalisation is valid,
and on held-out-like tiles it picks the dense raster propagation, which the
training report finds fastest on 511 of its 512 held-out tiles."""
import json
import os

import numpy as np

import synth
from oracle import features as OF
from oracle import mlp as OM

DATA = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1405_7958_gb300", "data")


def _load():
    return np.load(os.path.join(DATA, "picker_config4.npz"))


def test_picker_parameters_are_consistent():
    z = _load()
    assert z["master"].shape == (OM.NPARAM,) and z["wb"].shape == (OM.NPARAM,)
    assert z["m"].shape == (OM.NPARAM,) and z["v"].shape == (OM.NPARAM,)
    assert z["norm"].shape == (2 * OM.NIN,) and (z["norm"][OM.NIN:] > 0).all()
    assert int(z["step_count"]) > 0 and np.isfinite(z["master"]).all()
    u = z["master"].view(np.uint32).astype(np.uint64)
    rne = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint16)
    assert np.array_equal(rne, z["wb"].astype(np.uint16))


def test_picker_chooses_raster_on_held_out_like_tiles():
    z = _load()
    p = OM.bf16_bits_to_f64(z["wb"])
    for H, W, ns, seed in synth.batch_sizes(6, 424242, 1024, 1536, 256):
        f = OF.features(synth.tile(H, W, seed, ns))
        logits = OM.forward(p, z["norm"], f[None, :])[3][0]
        assert int(np.argmax(logits)) == 0, (H, W, ns, logits)


def test_training_report_matches_its_counts():
    with open(os.path.join(DATA, "picker_config4_report.json")) as fh:
        r = json.load(fh)
    ev = r["eval"]
    assert sum(ev["pick_counts"].values()) == ev["tiles"] == sum(ev["best_counts"].values())
    assert ev["time_learned_ms"] >= ev["time_best_ms"] and ev["time_plain_ms"] >= ev["time_best_ms"]
    assert 0.0 <= ev["accuracy"] <= 1.0 and ev["regret_mean_ms"] >= 0.0
