"""Host logic of the tuning pipeline (paper_1804_10694_gb300/tune.py), on the
CPU: the autotuner times one representative of each effective
configuration of a shape, and tune.py maps any candidate onto the timed
representative by its effective key.  That key must split the candidates
exactly as the library's cost-model features do -- candidates with one key
look identical to the model, candidates with different keys differ -- or
the regret reported for a pick would be the time of another kernel."""
import numpy as np

import paper_1804_10694_gb300 as pkg
from paper_1804_10694_gb300 import tune


def test_effective_key_partitions_like_the_model_features():
    rng = np.random.default_rng(9)
    shapes = [tuple(int(x) for x in 2 ** rng.uniform(5, 14, 3)) for _ in range(25)]
    shapes += [(1060, 1060, 1060), (8192, 8192, 8192), (50176, 64, 576), (1, 300, 7)]
    for mode in ("bf16x3", "tf32x3", "bf16x6"):
        for M, N, K in shapes:
            groups = {}
            for cid in range(pkg.config_count(mode)):
                key = tune.effective_key(mode, cid, M, N, K)
                feats = tuple(pkg.costmodel_features(M, N, K, mode, cid).tolist())
                groups.setdefault(key, set()).add(feats)
            # one feature vector per key ...
            assert all(len(f) == 1 for f in groups.values()), (mode, M, N, K)
            # ... and a different one for every key
            vecs = [next(iter(f)) for f in groups.values()]
            assert len(set(vecs)) == len(vecs), (mode, M, N, K)


def test_timed_choice_maps_onto_the_timed_representative():
    M, N, K = 1060, 1060, 1060
    mode = "bf16x3"
    reps = {}
    for cid in range(pkg.config_count(mode)):
        reps.setdefault(tune.effective_key(mode, cid, M, N, K), cid)
    times = {cid: float(i + 1) for i, cid in enumerate(reps.values())}
    for cid in range(pkg.config_count(mode)):
        rep = reps[tune.effective_key(mode, cid, M, N, K)]
        assert tune.timed_choice(times, mode, cid, (M, N, K)) == times[rep]
