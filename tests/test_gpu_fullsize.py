"""Full-size workloads through the launch configuration the bench times.

Each database is generated at its full size and scored by graph-captured
batched plans (one per filter); the oracle then checks, one sequence at a
time, a sample of the outputs: the longest and shortest sequences, planted
ones where the workload has them, and random ones.  Bit-exact.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1707_09683_gb300 import build, mpf, synth

pytestmark = pytest.mark.gpu


def sample_index(db, rng, planted=None, n_random=600, n_edge=60):
    order = np.argsort(db.lengths, kind="stable")
    pick = [order[:n_edge], order[-n_edge:], rng.choice(db.n_seqs, n_random, replace=False)]
    if planted is not None and planted.size:
        pick.append(rng.choice(planted, min(planted.size, 300), replace=False))
    return np.unique(np.concatenate(pick)).astype(np.uint64)


def run_and_check(wl, queries, rng, planted=None):
    ctx = mpf.Context(0)
    db = mpf.Database(ctx, wl.db.residues, wl.db.offsets, wl.db.lengths)
    profs = [mpf.Profile(ctx, wl.profiles[i]) for i in queries]
    n, q = db.n_seqs, len(profs)
    dev = torch.device("cuda", 0)
    idx = sample_index(wl.db, rng, planted)
    n_flag = 0
    for gf, of in ((mpf.MSV, oracle.MSV), (mpf.SSV, oracle.SSV)):
        raw = torch.empty(q * n, dtype=torch.uint8, device=dev)
        flag = torch.empty(q * n, dtype=torch.uint8, device=dev)
        nat = torch.empty(q * n, dtype=torch.float32, device=dev)
        plan = mpf.Plan(ctx, gf, profs, db, raw, flag, nat)
        plan.capture_graph()
        plan.launch()
        ctx.sync()
        raw_h, flag_h, nat_h = raw.cpu().numpy(), flag.cpu().numpy(), nat.cpu().numpy()
        plan.close()
        for j, i in enumerate(queries):
            exp = oracle.scan(of, wl.profiles[i], wl.db.residues, wl.db.offsets, wl.db.lengths,
                              index=idx, nthreads=16)
            sel = j * n + idx.astype(np.int64)
            assert np.array_equal(raw_h[sel], exp[0]), (wl.name, gf, i)
            assert np.array_equal(flag_h[sel], exp[1]), (wl.name, gf, i)
            assert np.array_equal(nat_h[sel].view(np.uint32), exp[2].view(np.uint32)), (wl.name, gf, i)
            n_flag += int(exp[1].sum())
    for p in profs:
        p.close()
    db.close()
    ctx.close()
    return n_flag


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    oracle.build()


def test_model_length_sweep_full_database():
    wl = synth.make_workload(1)
    run_and_check(wl, list(range(len(wl.profiles))), np.random.default_rng(11))


def test_overflow_batch_full_database():
    wl = synth.make_workload(2)
    rng = np.random.default_rng(12)
    queries = sorted(rng.choice(len(wl.profiles), 8, replace=False).tolist())
    assert run_and_check(wl, queries, rng, planted=wl.planted) > 0


def test_throughput_workload_full_database():
    wl = synth.make_workload(4, n_queries=12)
    run_and_check(wl, list(range(12)), np.random.default_rng(13))
