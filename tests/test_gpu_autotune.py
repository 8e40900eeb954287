"""The autotuner times built configurations on the device, keeps the
fastest, and the tuned profile still scores exactly like the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1707_09683_gb300 import autotune, build, mpf, synth

pytestmark = pytest.mark.gpu


def test_autotune_picks_a_candidate_and_keeps_parity(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    wl = synth.make_workload(1, n_seqs=20000)
    ctx = mpf.Context(0)
    db = mpf.Database(ctx, wl.db.residues, wl.db.offsets, wl.db.lengths)
    cache = str(tmp_path / "tune.json")
    tuner = autotune.Autotuner(ctx, db, cache_path=cache, reps=2)
    for rec in (wl.profiles[1], wl.profiles[3]):          # M = 100, 400
        prof = mpf.Profile(ctx, rec)
        for filt, of in ((mpf.SSV, oracle.SSV), (mpf.MSV, oracle.MSV)):
            cfg = tuner.tune(prof, filt)
            assert cfg in autotune.candidates(rec.M)
            assert prof.get_config(filt) == cfg
            times = tuner.timings[tuner.key(filt, rec.M)]
            configs = {k: v for k, v in times.items() if "/" not in k}
            shared = prof.get_table_memory(filt) == mpf.TABLE_SHARED and cfg[0] == 32 and \
                f"{cfg[0]}x{cfg[1]}s" in configs
            best = f"{cfg[0]}x{cfg[1]}" + ("s" if shared else "")
            assert min(configs.values()) == times[best]
            factor = prof.get_shard_factor(filt)
            shard_t = {1: times[best]}
            shard_t.update({int(k.split("/")[1]): v for k, v in times.items() if k.startswith(best + "/")})
            assert set(shard_t) == set(autotune.SHARD_FACTORS)
            assert shard_t[factor] == min(shard_t.values())
            n = db.n_seqs
            raw, flag = np.empty(n, np.uint8), np.empty(n, np.uint8)
            (mpf.ssv_scan if filt == mpf.SSV else mpf.msv_scan)(ctx, prof, db, raw, flag)
            exp = oracle.scan(of, rec, wl.db.residues, wl.db.offsets, wl.db.lengths,
                              index=np.arange(0, n, 7, dtype=np.uint64), nthreads=8)
            assert np.array_equal(raw[::7], exp[0]) and np.array_equal(flag[::7], exp[1])
        prof.close()
    tuner.save()
    again = autotune.Autotuner(ctx, db, cache_path=cache)
    assert again.table == tuner.table


def test_tuned_configurations_mixed_in_one_batch_match_the_oracle():
    """Queries shaped like the 64-query workload (M uniform in [50, 2500],
    planted segments), each tuned on the database -- lanes and words, shared
    or tensor-memory table, shard factor -- then scored together by one
    graph-captured batched plan per filter: every output equals the oracle."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    oracle.build()
    wl = synth.make_workload(2, n_seqs=12000, n_queries=6)
    ctx = mpf.Context(0)
    db = mpf.Database(ctx, wl.db.residues, wl.db.offsets, wl.db.lengths)
    tuner = autotune.Autotuner(ctx, db, reps=1)
    profs = [mpf.Profile(ctx, p) for p in wl.profiles]
    for pr in profs:
        for filt in (mpf.MSV, mpf.SSV):
            tuner.tune(pr, filt)
    n, q = db.n_seqs, len(profs)
    dev = torch.device("cuda", 0)
    for filt, of in ((mpf.MSV, oracle.MSV), (mpf.SSV, oracle.SSV)):
        outs = [torch.empty(q * n, dtype=t, device=dev) for t in (torch.uint8, torch.uint8, torch.float32)]
        plan = mpf.Plan(ctx, filt, profs, db, *outs)
        plan.capture_graph()
        plan.launch()
        ctx.sync()
        got = [t.cpu().numpy() for t in outs]
        plan.close()
        for i, rec in enumerate(wl.profiles):
            exp = oracle.scan(of, rec, wl.db.residues, wl.db.offsets, wl.db.lengths, nthreads=8)
            sl = slice(i * n, (i + 1) * n)
            assert np.array_equal(got[0][sl], exp[0]) and np.array_equal(got[1][sl], exp[1]), (rec.M, filt)
            assert np.array_equal(got[2][sl].view(np.uint32), exp[2].view(np.uint32)), (rec.M, filt)
    for pr in profs:
        pr.close()
    db.close()
    ctx.close()
