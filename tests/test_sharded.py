"""The sharded update (paper_2512_16642_gb300.sharded) on the GPU, through the C ABI: all ranks'
shards in one process on one device, one after another (the exchange and the sums as local copies
and additions; no kernel of one rank waits for another's), against the unsharded update on the
same inputs.  Every frequency's Hessian is computed from the same transforms in the same order,
so the Hessians and factors agree bit for bit; the multipliers differ only by the order of the sum
over frequencies in the synthesis."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.mark.parametrize("world,precision", [(2, 0), (3, 0), (2, 1), (3, 1)])
def test_sharded_update_equals_unsharded(world, precision):
    import torch

    from paper_2512_16642_gb300 import egh, sharded

    c = synth.case_small()
    geom = {k: c[k] for k in ("nz", "nx", "dz", "dx", "nsponge", "sponge_R", "dt", "nt", "rec_iz",
                              "rec_ix", "freqs")}
    kw = {"precision": precision, "gram_splits": 4}
    vel = torch.from_numpy(np.float32(c.vel_start)).cuda()
    rng = np.random.default_rng(8)
    resid = torch.from_numpy(synth.bandlimited_noise(rng, (6, c.rec_ix.size, c.nt), c.dt, 2.0, 10.0)
                             .astype(np.float32)).cuda()
    with egh.Context(*(geom[k] for k in ("nz", "nx", "dz", "dx", "nsponge", "sponge_R", "dt", "nt",
                                         "rec_iz", "rec_ix", "freqs")), **kw) as ctx:
        ctx.green(vel)
        mu_ref = ctx.hessian(egh.EGH_MU_REL_MEANDIAG, c.mu_alpha)
        Q_ref = ctx.get_hessian(False)
        ctx.factor()
        L_ref = ctx.get_hessian(True)
        m_ref = torch.empty_like(resid)
        ctx.deblur(resid, m_ref)
    shards = [sharded.Shard(geom, r, world, **kw) for r in range(world)]
    try:
        mult = torch.empty_like(resid)
        mu = sharded.update_in_process(shards, vel, resid, mult, c.mu_alpha)
        assert mu == pytest.approx(mu_ref, rel=1e-12)
        for s in shards:
            k0, k1 = s.kb[s.rank]
            assert np.array_equal(s.hess_ctx.get_hessian(False), Q_ref[k0:k1]), s.rank
            assert np.array_equal(s.hess_ctx.get_hessian(True), L_ref[k0:k1]), s.rank
            r0, r1 = s.rb[s.rank]
            assert s.green_ctx.stats()["pde_solves"] == r1 - r0
        torch.cuda.synchronize()
        assert rel(mult.cpu().numpy(), m_ref.cpu().numpy()) <= 1e-6
    finally:
        for s in shards:
            s.close()
