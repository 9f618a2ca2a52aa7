"""Serving loop (egh_server_*): continuous batching of deblur requests against resident factored
Hessian sets, through the C ABI.

Each request's multipliers are checked against the FP64 oracle (Cholesky of the same Hessian,
transform, solve, synthesis), and against the same request run alone: a request's sources are
its own right-hand sides, so its result does not depend on what it is batched or overlapped
with.  Admission keeps the device buffers inside the HBM budget; a request larger than the
budget is refused at submission.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

MULT_TOL = 1e-3


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _hpd_set(rng, nrec, nf):
    """Seeded synthetic Hermitian positive-definite Hessians Q_k = A A^H / m + mu I (complex64),
    frequencies evenly spaced in 2-10 Hz."""
    m = 2 * nrec
    A = (rng.standard_normal((nf, nrec, m)) + 1j * rng.standard_normal((nf, nrec, m))) / np.sqrt(m)
    Q = A @ A.conj().transpose(0, 2, 1)
    Q += 0.05 * np.mean(np.einsum("kii->ki", Q).real) * np.eye(nrec)
    Q = 0.5 * (Q + Q.conj().transpose(0, 2, 1))
    return Q.astype(np.complex64), np.linspace(2.0, 10.0, nf)


def _pinned(shape, torch, fill=None):
    t = torch.empty(shape, dtype=torch.float32, pin_memory=True)
    if fill is not None:
        t.copy_(torch.from_numpy(np.ascontiguousarray(fill, np.float32)))
    return t


def _requests(rng, sets, n):
    out = []
    for _ in range(n):
        sid = int(rng.integers(len(sets)))
        ns = int(rng.integers(1, 10))
        nt_d = int(rng.integers(256, 700))  # long enough for several 2-10 Hz bins
        nrec = sets[sid][0].shape[1]
        out.append((sid, synth.bandlimited_noise(rng, (ns, nrec, nt_d), 1e-3, 2.0, 10.0)))
    return out


@pytest.mark.parametrize("precision", [0, 1])
def test_alone_equals_mix_and_oracle(precision):
    import torch
    from paper_2512_16642_gb300 import egh

    rng = np.random.default_rng(41 + precision)
    sets = [_hpd_set(rng, nrec, nf) for nrec, nf in ((8, 3), (13, 5), (21, 7))]
    reqs = _requests(rng, sets, 14)
    dt, nt_record, max_nt = 1e-3, 1000, 1024
    with egh.Server(256 << 20, slots=4, max_batch_sources=24, precision=precision) as sv:
        ids = [sv.add_set(Q, f, dt, nt_record, max_nt) for Q, f in sets]
        ins = [_pinned(r.shape, torch, r) for _, r in reqs]
        alone = []
        for (sid, r), rin in zip(reqs, ins):
            out = _pinned(r.shape, torch)
            sv.wait(sv.submit(ids[sid], rin, out))
            alone.append(out.numpy().copy())
        # the same requests all at once, in a shuffled order: batched and overlapped.  Admission
        # is held while they are submitted so that they queue together whatever the host's timing
        outs = [_pinned(r.shape, torch) for _, r in reqs]
        order = rng.permutation(len(reqs))
        sv.reset_stats()
        sv.hold(True)
        rids = {i: sv.submit(ids[reqs[i][0]], ins[i], outs[i]) for i in order}
        assert sv.stats()["completed"] == 0
        sv.hold(False)
        for i in order:
            sv.wait(rids[i])
        st = sv.stats()
    for i in range(len(reqs)):
        np.testing.assert_array_equal(outs[i].numpy(), alone[i])
    assert st["completed"] == len(reqs)
    assert st["batches"] < st["completed"]  # some requests shared a solve
    assert st["peak_bytes_in_use"] <= 256 << 20
    for i in range(len(reqs)):
        sid, r = reqs[i]
        Q, f = sets[sid]
        L = oracle.cholesky(Q.astype(np.complex128))
        m = oracle.deblur(L, r.astype(np.float32).astype(np.float64), f, dt, nt_ref=nt_record)[0]
        assert rel(alone[i], m) <= MULT_TOL, i


def test_admission_by_budget_and_overlap():
    import torch
    from paper_2512_16642_gb300 import egh

    rng = np.random.default_rng(7)
    Q, f = _hpd_set(rng, 64, 12)
    ns, nt_d = 16, 2000
    per_request = 2 * ns * 64 * nt_d * 4 + 12 * 64 * ns * 8  # in + out traces + spectra
    budget = int(2.5 * per_request) + (1 << 20)
    with egh.Server(budget, slots=8, max_batch_sources=ns, precision=0) as sv:
        sid = sv.add_set(Q, f, 1e-3, 4000, 4096)
        big = _pinned((200, 64, 4000), torch)
        with pytest.raises(egh.EghError) as ei:
            sv.submit(sid, big, big)
        assert ei.value.status == egh.EGH_ENOMEM
        r = synth.bandlimited_noise(rng, (ns, 64, nt_d), 1e-3, 2.0, 10.0)
        rin = _pinned(r.shape, torch, r)
        outs = [_pinned(r.shape, torch) for _ in range(10)]
        rids = [sv.submit(sid, rin, o) for o in outs]
        for rid in rids:
            assert sv.wait(rid) > 0.0
        st = sv.stats()
        assert st["completed"] == 10 and st["rejected"] == 1
        assert st["peak_bytes_in_use"] <= budget
        assert 1 <= st["peak_in_flight"] <= 2  # the budget holds two requests at a time
        for o in outs[1:]:
            np.testing.assert_array_equal(o.numpy(), outs[0].numpy())
    with egh.Server(64 * per_request, slots=8, max_batch_sources=ns, precision=0) as sv:
        sid = sv.add_set(Q, f, 1e-3, 4000, 4096)
        sv.hold(True)  # queued together, so that the admissions follow each other at once
        rids = [sv.submit(sid, rin, o) for o in outs]
        sv.hold(False)
        sv.drain()
        for rid in rids:
            sv.wait(rid)
        assert sv.stats()["peak_in_flight"] >= 2  # batches overlapped on the device


@pytest.mark.parametrize("precision", [0, 1])
def test_full_size_set_sampled(precision):
    """The largest set of the benchmark's serving mix (461 receivers, 40 frequencies 2-10 Hz) and
    its largest request (64 sources x 4000 samples) in the launch configuration the benchmark
    times; the multipliers of sampled sources against the FP64 oracle (sources are independent
    right-hand sides, so the oracle solves only the sampled ones)."""
    import torch
    from paper_2512_16642_gb300 import egh

    rng = np.random.default_rng(77)
    Q, f = _hpd_set(rng, 461, 40)
    ns, nt_d, dt = 64, 4000, 1e-3
    r = synth.bandlimited_noise(rng, (ns, 461, nt_d), dt, 2.0, 10.0)
    sample = np.array([0, 37, 63])
    L = oracle.cholesky(Q.astype(np.complex128))
    ref = oracle.deblur(L, r[sample].astype(np.float32).astype(np.float64), f, dt, nt_ref=4000)[0]
    with egh.Server(8 << 30, slots=4, max_batch_sources=128, precision=precision) as sv:
        sid = sv.add_set(Q, f, dt, 4000, 4096)
        rin = _pinned(r.shape, torch, r)
        out = _pinned(r.shape, torch)
        sv.wait(sv.submit(sid, rin, out))
    got = out.numpy()[sample]
    for i in range(sample.size):
        assert rel(got[i], ref[i]) <= MULT_TOL, (precision, int(sample[i]))


@pytest.mark.parametrize("nt_d", [1200, 1001])
def test_many_frequencies(nt_d):
    """60 frequencies (the tensor-core transform's widest component block, 2 nf up to 128),
    a trace length that is and one that is not a multiple of four, against the FP64 oracle."""
    import torch
    from paper_2512_16642_gb300 import egh

    rng = np.random.default_rng(5 + nt_d)
    Q, f = _hpd_set(rng, 37, 60)
    r = synth.bandlimited_noise(rng, (3, 37, nt_d), 1e-3, 2.0, 10.0)
    L = oracle.cholesky(Q.astype(np.complex128))
    ref = oracle.deblur(L, r.astype(np.float32).astype(np.float64), f, 1e-3, nt_ref=2000)[0]
    with egh.Server(1 << 30, slots=2, max_batch_sources=8, precision=1) as sv:
        sid = sv.add_set(Q, f, 1e-3, 2000, 2048)
        rin = _pinned(r.shape, torch, r)
        out = _pinned(r.shape, torch)
        sv.wait(sv.submit(sid, rin, out))
    assert rel(out.numpy(), ref) <= MULT_TOL


def test_bounded_wait_expiry_fails_only_its_request():
    """A batch whose forward transform has a bounded device wait run out (test hook: one block
    waits on an mbarrier that nothing signals, about 0.2 ms) fails its own requests with
    EGH_ETIMEOUT through egh_server_wait, and only those: the next request gets the multipliers
    of a clean run bit for bit, the server stays usable, and the next drain reports that a wait
    ran out since the previous drain (and the one after it does not)."""
    import torch
    from paper_2512_16642_gb300 import egh

    rng = np.random.default_rng(77)
    Q, f = _hpd_set(rng, 11, 4)
    r = synth.bandlimited_noise(rng, (3, 11, 400), 1e-3, 2.0, 10.0)
    with egh.Server(64 << 20, slots=2, max_batch_sources=8, precision=1) as sv:
        sid = sv.add_set(Q, f, 1e-3, 1000, 512)
        rin = _pinned(r.shape, torch, r)
        ref = _pinned(r.shape, torch)
        sv.wait(sv.submit(sid, rin, ref))
        sv.drain()
        sv.test_expire_wait(1)
        bad = _pinned(r.shape, torch)
        rid = sv.submit(sid, rin, bad)
        with pytest.raises(egh.EghError) as ei:
            sv.wait(rid)
        assert ei.value.status == egh.EGH_ETIMEOUT and "bounded device wait" in str(ei.value)
        with pytest.raises(egh.EghError):  # the id was released with its status
            sv.wait(rid)
        out = _pinned(r.shape, torch)
        sv.wait(sv.submit(sid, rin, out))
        assert np.array_equal(out.numpy(), ref.numpy())
        with pytest.raises(egh.EghError) as ei:
            sv.drain()
        assert ei.value.status == egh.EGH_ETIMEOUT
        sv.drain()
        st = sv.stats()
        assert st["completed"] == 3


@pytest.mark.parametrize("nrec,nf,ns,nt_d", [
    (13, 5, 3, 4),          # one stage: clusters of one CTA
    (21, 20, 23, 132),      # three stages (clusters of two), four ragged trace tiles
    (21, 20, 1220, 300),    # 201 trace tiles: several per cluster; units across tile ends
    (9, 12, 5, 8192),       # 128 stages: clusters of eight, two TMEM blocks per rank and tile
    (9, 40, 7, 1028),       # 40 frequencies: 128-sample synthesis units, a 4-sample last one
    (21, 26, 115, 4000),    # the benchmark's frequencies and trace length
])
def test_persistent_transforms_shapes(nrec, nf, ns, nt_d):
    """The persistent forward transform (TMA stages, time axis split over a cluster, partials
    summed by the owning rank through distributed shared memory) and the persistent synthesis
    (TMA stores) on device buffers, at shapes that reach each of their edge cases, against the
    FP64 oracle's transform, Cholesky solve and synthesis of the same Hessians."""
    import torch
    from paper_2512_16642_gb300 import egh

    rng = np.random.default_rng(1000 + nt_d + ns)
    Q, f = _hpd_set(rng, nrec, nf)
    dt = 1e-3
    nt_record = max(nt_d, 256)
    # white residuals: every sample counts, however short the trace
    r = rng.standard_normal((ns, nrec, nt_d)).astype(np.float32)
    L = oracle.cholesky(Q.astype(np.complex128))
    ref = oracle.deblur(L, r.astype(np.float64), f, dt, nt_ref=nt_record)[0]
    with egh.Server(1 << 30, slots=2, max_batch_sources=2048, precision=1) as sv:
        sid = sv.add_set(Q, f, dt, nt_record, max(nt_d, 1024))
        rin = _pinned(r.shape, torch, r)
        out = _pinned(r.shape, torch)
        sv.wait(sv.submit(sid, rin, out))
        # a subset of the sources alone: fewer trace tiles, the same arithmetic per trace
        sub = slice(ns // 2, ns // 2 + 2)
        rsub = _pinned(r[sub].shape, torch, r[sub])
        osub = _pinned(r[sub].shape, torch)
        sv.wait(sv.submit(sid, rsub, osub))
    got = out.numpy()
    assert np.all(np.isfinite(got))
    assert np.array_equal(osub.numpy(), got[sub])
    assert rel(got, ref) <= MULT_TOL
    for s in range(0, ns, max(1, ns // 7)):
        assert rel(got[s], ref[s]) <= MULT_TOL, s
