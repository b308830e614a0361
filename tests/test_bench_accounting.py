"""Host-side accounting of bench.py (no GPU): the algorithmic bytes behind the
roofline fraction, and the provenance of the DRAM traffic figures.

A blend reads 28 bytes per slot for the softmax rgb blend (face id, depth,
three barycentrics, distance) and 12 for the silhouette (face id and
distance only); the forward always writes all 28.  Every measured traffic
figure names the committed profile summary it was taken from.
"""
import dataclasses
import os

import pytest

import bench
from paper_2007_08501_gb300 import workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("index", [1, 4])
def test_algorithmic_bytes_per_slot(index):
    w = workloads.workload(index)
    b = w.batch
    slots = b.N * w.image_size * w.image_size * w.K
    alg = bench.algorithmic_bytes(w)
    # the slot-proportional part of each stage, with the mesh and image terms removed
    alg1 = bench.algorithmic_bytes(dataclasses.replace(w, K=w.K + 1))
    per_slot = {k: (alg1[k] - alg[k]) * w.K / slots for k in alg}
    read = 12 if w.blend_mode == "sil" else 28
    assert per_slot["fwd"] == pytest.approx(28)
    assert per_slot["rast_fwd"] == pytest.approx(28)
    assert per_slot["bwd"] == pytest.approx(read)
    assert per_slot["blend_fwd"] == pytest.approx(read)
    assert per_slot["blend_bwd"] == pytest.approx(read + 20)


def test_traffic_figures_name_committed_profiles():
    for key, entry in bench.TRAFFIC_BYTES.items():
        assert entry["bytes"] > 0, key
        path = entry["profile"].split(" ")[0]
        assert os.path.isfile(os.path.join(ROOT, path)), (key, path)
