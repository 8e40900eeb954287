"""The debug build's kernel index checks (libmpf_debug.so).

Every kernel family runs on the debug library over inputs that exercise its
ragged edges -- striped scans in every lane-group size (and through the
allocation-free entry point), packed sets of queries sharing a warp's
sequence, both filters from one sweep (striped, packed and tiled), rank lists from the
SSV -> MSV hand-off, long models through the tiled kernels (with the MSV
fallback list) and the lane-segment kernel with 16-bit and byte rows, the
Viterbi kernels and variants (rows in shared or device memory), the MSV ->
Viterbi stage -- and no check may fire (mpf_sync would raise MPF_EDEVICE);
results are compared with the oracle.
The self-test shows a failed check reaching mpf_sync as MPF_EDEVICE.  The
debug library runs in a child process so it never mixes with the release
library the other tests load.
"""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1707_09683_gb300 import build

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys
sys.path.insert(0, ROOT)
import numpy as np
import torch
import oracle
from paper_1707_09683_gb300 import mpf, synth

mpf.load(mpf.DEBUG_LIB_PATH)
dev = torch.device("cuda", 0)

def same(a, b):
    return np.array_equal(np.asarray(a).view(np.uint8), np.asarray(b).view(np.uint8))

# The self-test: a failing check is reported, on a context of its own.
c0 = mpf.Context(0)
mpf.debug_check_selftest(c0)
try:
    c0.sync()
    raise SystemExit("self-test check was not reported")
except mpf.MpfError as e:
    assert e.status == mpf.MPF_EDEVICE, e.status
c0.close()

ctx = mpf.Context(0)
rng = np.random.default_rng(5)
wl = synth.make_workload(0, n_seqs=700)
dbh = wl.db
db = mpf.Database(ctx, dbh.residues, dbh.offsets, dbh.lengths)
n = db.n_seqs

# Striped scans in every lane-group size, both filters, and long models.
for M, lanes, words in ((48, 1, 24), (100, 2, 26), (100, 4, 14), (300, 8, 20), (700, 16, 22),
                        (2405, 32, 38), (3500, 0, 0), (31000, 0, 0)):
    rec = synth.make_profile(M, rng)
    p = mpf.Profile(ctx, rec)
    for gf, of in ((mpf.MSV, oracle.MSV), (mpf.SSV, oracle.SSV)):
        if lanes:
            p.set_config(gf, lanes, words)
        out = [torch.empty(n, dtype=t, device=dev) for t in (torch.uint8, torch.uint8, torch.float32)]
        mpf.scan_batch(ctx, gf, [p], db, *out)
        ctx.sync()
        idx = np.arange(0, n, 7, dtype=np.uint64)
        want = oracle.scan(of, rec, dbh.residues, dbh.offsets, dbh.lengths, index=idx, nthreads=8)
        for g, w in zip(out, want):
            assert same(g.cpu().numpy()[idx.astype(np.int64)], w), (M, gf)
    p.close()

# Packed sets: queries of 1 to 16 lanes sharing a warp's sequence (one set
# with an empty slot), in one plan per filter.
cfgs = [(1, 14)] * 27 + [(4, 26)] * 7 + [(8, 22)] * 4 + [(16, 18)] * 2
recs = [synth.make_profile(2 * l * w - 1, rng) for l, w in cfgs]
profs = [mpf.Profile(ctx, r) for r in recs]
for gf, of in ((mpf.MSV, oracle.MSV), (mpf.SSV, oracle.SSV)):
    for pr, (l, w) in zip(profs, cfgs):
        pr.set_config(gf, l, w)
    q = len(profs)
    out = [torch.empty(q * n, dtype=t, device=dev) for t in (torch.uint8, torch.uint8, torch.float32)]
    pl = mpf.Plan(ctx, gf, profs, db, *out)
    assert max(g["queries_per_warp"] for g in pl.groups()) == 32, pl.groups()
    pl.launch()
    ctx.sync()
    pl.close()
    idx = np.arange(0, n, 5, dtype=np.uint64)
    for i in (0, 26, 27, 33, 34, 38, 39):
        want = oracle.scan(of, recs[i], dbh.residues, dbh.offsets, dbh.lengths, index=idx, nthreads=8)
        for g, w in zip(out, want):
            got = g[i * n:(i + 1) * n].cpu().numpy()[idx.astype(np.int64)]
            assert same(got, w), ("packed", i, gf)
# Both filters in one sweep: the packed set above, whole-warp queries with
# the table in TMEM, and a long model (tiles in TMEM), in one plan.
recs2 = recs[27:38] + [synth.make_profile(M, rng) for M in (1500, 2405, 3500)]
profs2 = profs[27:38] + [mpf.Profile(ctx, r) for r in recs2[11:]]
q = len(profs2)
out = [torch.empty(2 * q * n, dtype=t, device=dev) for t in (torch.uint8, torch.uint8, torch.float32)]
pl = mpf.Plan(ctx, mpf.MSV_SSV, profs2, db, *out)
assert all(g["filters"] == 3 for g in pl.groups()), pl.groups()
pl.launch()
ctx.sync()
pl.close()
idx = np.arange(0, n, 5, dtype=np.uint64)
for fb, of in enumerate((oracle.MSV, oracle.SSV)):
    for i in (0, 7, 11, 12, 13):
        want = oracle.scan(of, recs2[i], dbh.residues, dbh.offsets, dbh.lengths, index=idx, nthreads=8)
        for g, w in zip(out, want):
            got = g[(fb * q + i) * n:(fb * q + i + 1) * n].cpu().numpy()[idx.astype(np.int64)]
            assert same(got, w), ("one sweep", i, fb)
for pr in profs + profs2[11:]:
    pr.close()

# The allocation-free entry point (its kernel reports through the context's
# status word too).
rec = synth.make_profile(300, rng)
p = mpf.Profile(ctx, rec)
lib = mpf.load()
for gf, of in ((mpf.MSV, oracle.MSV), (mpf.SSV, oracle.SSV)):
    out = [torch.empty(n, dtype=t, device=dev) for t in (torch.uint8, torch.uint8, torch.float32)]
    st = lib.mpf_scan_noalloc(ctx.handle, gf, p.handle, db.handle, *[t.data_ptr() for t in out])
    assert st == mpf.MPF_OK, st
    ctx.sync()
    want = oracle.scan(of, rec, dbh.residues, dbh.offsets, dbh.lengths, nthreads=8)
    for g, w in zip(out, want):
        assert same(g.cpu().numpy(), w), ("noalloc", gf)
p.close()

# The exact lane-segment MSV kernel with 16-bit and byte rows (profiles
# whose begin score cannot be held), and the tiled MSV pass handing planted
# hits to it through the fallback list.
pl_db = synth.make_database(300, 355, 10, 2000, rng)
pl_rec = synth.make_profile(3500, rng)
synth.plant_segments(pl_db, [pl_rec], 0.3, rng)
cases = [(synth.random_profile(3500, 20, rng, bias=250), dbh),
         (synth.random_profile(31000, 20, rng, bias=250), dbh),
         (pl_rec, pl_db)]
for rec, d in cases:
    dd = mpf.Database(ctx, d.residues, d.offsets, d.lengths)
    p = mpf.Profile(ctx, rec)
    m = dd.n_seqs
    out = [torch.empty(m, dtype=t, device=dev) for t in (torch.uint8, torch.uint8, torch.float32)]
    mpf.scan_batch(ctx, mpf.MSV, [p], dd, *out)
    ctx.sync()
    idx = np.arange(0, m, 7, dtype=np.uint64)
    want = oracle.scan(oracle.MSV, rec, d.residues, d.offsets, d.lengths, index=idx, nthreads=8)
    for g, w in zip(out, want):
        assert same(g.cpu().numpy()[idx.astype(np.int64)], w), rec.M
    p.close()
    dd.close()

# The SSV -> MSV hand-off (rank lists) with a striped and a long profile,
# then the MSV -> Viterbi stage.
wl2 = synth.make_workload(2, n_seqs=2000, n_queries=2)
db2 = mpf.Database(ctx, wl2.db.residues, wl2.db.offsets, wl2.db.lengths)
recs = [wl2.profiles[0], synth.make_profile(4000, rng)]
profs = [mpf.Profile(ctx, r) for r in recs]
m, q = db2.n_seqs, len(profs)
mk = lambda t: torch.empty(q * m, dtype=t, device=dev)
ssv_out = (mk(torch.uint8), mk(torch.uint8), mk(torch.float32))
msv_out = (mk(torch.uint8), mk(torch.uint8), mk(torch.float32))
n_pass = torch.empty(q, dtype=torch.int32, device=dev)
mpf.pipeline_scan(ctx, profs, db2, -5.0, ssv_out, msv_out, n_pass)
vrecs = [synth.make_vit_profile(r.M, rng) for r in recs]   # M = 4000: rows in device memory
vps = [mpf.VitProfile(ctx, v) for v in vrecs]
vs, vf, vn = mk(torch.int16), mk(torch.uint8), mk(torch.float32)
n2 = torch.empty(q, dtype=torch.int32, device=dev)
mpf.viterbi_rescore(ctx, vps, db2, msv_out[1], msv_out[2], -5.0, vs, vf, vn, n2)
ctx.sync()
for i, r in enumerate(recs):
    _, (mr, mf, mn), npass = oracle.pipeline(r, wl2.db.residues, wl2.db.offsets, wl2.db.lengths, -5.0,
                                             nthreads=8)
    sl = slice(i * m, (i + 1) * m)
    assert int(n_pass.cpu()[i]) == npass
    assert same(msv_out[0].cpu().numpy()[sl], mr) and same(msv_out[2].cpu().numpy()[sl], mn)
    want, nv = oracle.viterbi_stage(vrecs[i], wl2.db.residues, wl2.db.offsets, wl2.db.lengths, mf, mn,
                                    -5.0, nthreads=8)
    assert int(n2.cpu()[i]) == nv
    assert same(vs.cpu().numpy()[sl], want[0]) and same(vn.cpu().numpy()[sl], want[2])

# Viterbi kernels directly: fast (unroll 4 and 8, no D row) and general,
# with the rows in shared memory and (M > 3072) in device memory.
vrecs = [synth.make_vit_profile(M, rng) for M in (40, 700, 2600, 3500)]
vrecs.append(synth.random_vit_profile(150, 20, rng, lo=-500, hi=300))
vrecs.append(synth.random_vit_profile(3300, 20, rng, lo=-500, hi=300))
vps = [mpf.VitProfile(ctx, v) for v in vrecs]
q = len(vps)
vs, vf, vn = (torch.empty(q * n, dtype=t, device=dev) for t in (torch.int16, torch.uint8, torch.float32))
mpf.viterbi_scan(ctx, vps, db, vs, vf, vn)
ctx.sync()
for i, v in enumerate(vrecs):
    want = oracle.viterbi(v, dbh.residues, dbh.offsets, dbh.lengths, nthreads=8)
    sl = slice(i * n, (i + 1) * n)
    assert same(vs.cpu().numpy()[sl], want[0]) and same(vf.cpu().numpy()[sl], want[1])
print("OK")
""".replace("ROOT", repr(ROOT))


@pytest.fixture(scope="module")
def debug_lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    oracle.build()
    return build.build(debug=True)


def test_debug_build_reports_no_bad_index_and_matches_the_oracle(debug_lib):
    r = subprocess.run([sys.executable, "-c", SCRIPT], capture_output=True, text=True, timeout=1500)
    assert r.returncode == 0, (r.stdout[-2000:], r.stderr[-4000:])
    assert r.stdout.strip().endswith("OK")
