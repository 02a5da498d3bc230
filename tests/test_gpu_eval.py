"""GPU parity of the evaluation calls (Sect. VIII experiments) against the evaluation
oracle, on the filter's own cell estimates after a run over a seeded scene with ground
truth: cluster statistics within the fixed-point bound, Mahalanobis distances bit for bit
(binary32, same operation order) and the classification counts exactly."""
import numpy as np
import pytest

from oracle import eval_oracle as E
from paper_1605_02406_b300 import scene

pytestmark = pytest.mark.gpu


def _run(cfg, frames):
    from paper_1605_02406_b300.evaluate import Evaluator
    from paper_1605_02406_b300.filter import DogFilter
    seq = scene.frame_sequence_with_truth(cfg, frames, 1001)
    f = DogFilter(scene.filter_params(cfg))
    for grid, _ in seq:
        f.set_measurement_grid(**grid)
        f.step(cfg["dt"])
    truth = seq[-1][1]
    thr = np.concatenate([[0.0], np.logspace(-2, 3, 21)]).astype(np.float32)
    ev = Evaluator(f, len(truth["velocity"]), thr)
    return f, ev, truth, thr


@pytest.mark.parametrize("workload", ["plain_128", "automotive_1024"])
def test_eval_matches_oracle(workload):
    from paper_1605_02406_b300.evaluate import detections
    cfg = scene.CONFIGS[workload]
    f, ev, truth, thr = _run(cfg, 15 if workload == "plain_128" else 6)
    cells = f.cells()
    n_obj = len(truth["velocity"])
    st = ev.clusters(truth["object"])
    ref = E.cluster_stats(cells, truth["object"], n_obj)
    assert np.array_equal(st[:, 0], ref[:, 0])
    # fixed point 2^-32 per cell term, binary64 elsewhere
    assert np.allclose(st[:, 1:], ref[:, 1:], rtol=1e-9, atol=1e-8)
    hist, m = ev.classification(truth["dynamic"], 0.5)
    sel = ((truth["dynamic"] == 1) | (truth["dynamic"] == 2)) & (cells["m_occ"] >= np.float32(0.5))
    m_ref = E.mahalanobis0(cells["mean_vx"], cells["mean_vy"], cells["var_vx"], cells["var_vy"],
                           cells["cov_vxy"])
    assert np.array_equal(m[sel].view(np.uint32), m_ref[sel].view(np.uint32))
    assert np.all(m[~sel] == 0)
    assert np.array_equal(detections(hist), E.classify_counts(m_ref, truth["dynamic"], cells["m_occ"], 0.5, thr))
    assert hist[0].sum() > 0 and hist[1].sum() >= 0
    f.close()


def test_eval_rejects_bad_arguments():
    from paper_1605_02406_b300 import native as N
    from paper_1605_02406_b300.filter import DogFilter
    f = DogFilter(scene.filter_params(scene.CONFIGS["plain_128"]))
    with pytest.raises(N.DogError) as e:
        N.dog_eval_clusters(f.h, 0, 4, 0, 0)
    assert e.value.code == -1
    with pytest.raises(N.DogError) as e:
        N.dog_eval_mahalanobis(f.h, 16, 0.5, 16, 5000, 16, None)
    assert e.value.code == -7
    f.close()
