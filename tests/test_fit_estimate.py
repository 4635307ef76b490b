"""Host logic of the fitter of the built-in tile-choice estimate
(paper_1804_10694_gb300/fit_estimate.py), on the CPU.

The fitter searches the constants of the estimate that the library's default
tile choice uses (waves x (prologue + k-chunks a split x chunk cost +
epilogue) + split-K fix-up) for the least regret against timed
configurations.  Two things make its output usable: its estimate must be
the library's (with the library's constants it picks the library's default
configuration), and on timings that the estimate itself explains exactly it
must reach zero regret, starting from constants that do not."""
import itertools
import json
import random

import numpy as np

import paper_1804_10694_gb300 as pkg
from paper_1804_10694_gb300 import fit_estimate as fe

MODES = {2: "bf16x3", 3: "tf32x3", 4: "bf16x6"}
# the constants compiled into the library's default_config
SHIPPED = dict(chunk128=1.5, chunk_pair=2.0, epi64=3.3, epi128=7.2, epi_pair=28.8, a0=3.6,
               fix0=4.0, fix1=0.99, six=1.6)
# planted constants for synthetic timings (values of the fitter's search grid)
PLANTED = dict(chunk128=1.7, chunk_pair=2.5, epi64=2, epi128=4, epi_pair=16, a0=4, fix0=2,
               fix1=0.25, six=2.0)


def _shapes(n, seed):
    rng = np.random.default_rng(seed)
    return [tuple(int(x) for x in 2 ** rng.uniform(5, 13, 3)) for _ in range(n)]


def test_pick_is_the_library_default():
    """With the library's constants, the fitter's estimate picks the
    library's default configuration (every field) in every mode."""
    shapes = _shapes(150, 1) + [(n, n, n) for n in (128, 512, 1024, 1060, 4099, 8192)]
    shapes += [(50176, 64, 576), (12544, 128, 1152), (3136, 256, 2304)]
    for mode, name in MODES.items():
        for M, N, K in shapes:
            c = pkg.config_get(name, pkg.config_default(name, M, N, K))
            lib = (c["block_n"], c["split_k"], c["kb"], c["group_m"], c["fused"], c["cluster"])
            assert fe.pick(M, N, K, mode, SHIPPED) == lib, (name, M, N, K)


def _planted_csv(path, shapes):
    """Autotuner-format rows whose times are the estimate under PLANTED,
    for every packed candidate of every shape and mode."""
    k = PLANTED
    cols = "M,N,K,lda,ldb,ldc,mode,config_id,median_ms,block_n,split_k,kb,group_m,fused,cluster"
    lines = [cols]
    for mode in MODES:
        for M, N, K in shapes:
            chunks = fe.chunks_of(K, mode)
            cands = ((64, 1, 1.0, k["epi64"]), (128, 1, k["chunk128"], k["epi128"]),
                     (256, 2, k["chunk_pair"], k["epi_pair"]))
            for bn, cl, tc, te in cands:
                tiles = -(-M // (128 * cl)) * -(-N // bn)
                for sk in fe.SPLITS:
                    if sk > 1 and sk > chunks:
                        break
                    per = -(-chunks // sk)
                    eff = -(-chunks // per)
                    t = -(-(tiles * eff) // (152 // cl)) * (k["a0"] + per * tc * (k["six"] if mode == 4 else 1.0) + te)
                    if eff > 1:
                        t += k["fix0"] + k["fix1"] * M * N * eff * 1e-6
                    kb = 8 if (mode == 4 and cl == 2) else 4
                    lines.append(f"{M},{N},{K},{K},{N},{N},{mode},-1,{t!r},{bn},{sk},{kb},16,0,{cl}")
    path.write_text("\n".join(lines) + "\n")


def test_fit_reaches_zero_regret_on_timings_the_estimate_explains(tmp_path, capsys):
    path = tmp_path / "planted.csv"
    _planted_csv(path, _shapes(40, 3))
    table = fe.load([str(path)])
    assert len(table) == 40 * len(MODES)
    for mode in MODES:
        assert fe.regret(table, PLANTED, mode) == (0.0, 40)
    # the search's first draw and the shipped constants do not explain them
    grid = dict(chunk128=[1.3, 1.5, 1.7, 1.9], chunk_pair=[2.0, 2.5, 3.0, 3.5], epi64=[1, 2, 3, 4, 6],
                epi128=[2, 4, 6, 8, 12], epi_pair=[8, 16, 24, 32, 48], a0=[2, 4, 8, 12, 16],
                fix0=[0, 2, 4, 8], fix1=[0, 0.1, 0.25, 0.5, 1], six=[1.5, 2.0])
    combos = list(itertools.product(*(grid[name] for name in fe.KEYS)))
    random.Random(3).shuffle(combos)
    first = dict(zip(fe.KEYS, combos[0]))
    assert sum(fe.regret(table, first, m)[0] for m in MODES) > 0.05
    assert sum(fe.regret(table, SHIPPED, m)[0] for m in MODES) > 0.0
    k = fe.fit(table, samples=300, seed=3)
    for mode in MODES:
        assert fe.regret(table, k, mode) == (0.0, 40), (mode, k)
    # the command line prints the constants and the regret of each mode
    fe.main([str(path), "--samples", "300", "--heldout", str(path)])
    out = capsys.readouterr().out.splitlines()
    assert set(json.loads(out[0])) == set(fe.KEYS)
    assert any(line.startswith("bf16x6: train regret 0.0000, held-out 0.0000") for line in out)
