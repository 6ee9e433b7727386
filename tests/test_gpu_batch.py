"""The batched persistent launch (pp_batch_run) against the single-molecule path.

Each molecule of a batch must come out bit-identical to pp_make_ff +
pp_relax_scan (fused df) run on that molecule alone: the batch runs the same
FF pair-sum core and the same FIRE core, only scheduled differently.  The
single-molecule path is itself parity-tested against the FP64 oracle.
Also: CUDA-graph replay, a forced timeout of the bounded wait (reported as a
status, the context stays usable), and invalid descriptors being skipped.
"""
import copy
import ctypes

import numpy as np
import pytest
import torch

from helpers import case32
from paper_2401_14564_gb300 import afm, batch, pp, synth

pytestmark = pytest.mark.gpu


def cases(n=10, first_seed=1000):
    cs = [case32(c) for c in synth.batch_cases(n, first_seed)]
    # ragged extras: a scan that is not a multiple of the 8x4 tile, and a molecule without atoms
    r = copy.deepcopy(cs[0])
    r["scan"] = dict(r["scan"], nx=13, ny=7)
    cs.append(r)
    e = copy.deepcopy(cs[1])
    for k in ("x", "y", "z", "R", "eps", "q"):
        e["atoms"][k] = e["atoms"][k][:0]
    cs.append(e)
    return cs


def single(c):
    sim = afm.Simulator(c)
    sim.run(afm.atoms_to_device(c["atoms"]))
    torch.cuda.synchronize()
    g = c["grid"]
    return {"fz": sim.fz.cpu().numpy(), "df": sim.df.cpu().numpy(), "iters": sim.iters.cpu().numpy(),
            "pos": sim.pos.cpu().numpy(), "ff": sim.ff.view(g["nz"], g["ny"], g["nx"], 4).cpu().numpy()}


def test_batch_matches_single_molecule_path_bit_for_bit():
    cs = cases()
    b = batch.Batch(cs, want_pos=True)
    b.run()
    st, flags = b.status()
    assert st == 0 and flags == 0
    for n, c in enumerate(cs):
        got = {k: v.cpu().numpy() for k, v in b.molecule(n).items()}
        ref = single(c)
        for k in ("ff", "fz", "df", "iters", "pos"):
            assert np.array_equal(got[k], ref[k]), (n, k)


def test_forces_only_batch_matches_the_full_one():
    # ff_forces_only: the grids' forces and every scan output are bit for bit the full batch's,
    # the E slots are 0
    cs = cases(6, 3000)
    full, fo = batch.Batch(cs, want_pos=True), batch.Batch(cs, want_pos=True, ff_energy=False)
    full.run()
    fo.run()
    assert full.status() == (0, 0) and fo.status() == (0, 0)
    for n in range(len(cs)):
        a, b = full.molecule(n), fo.molecule(n)
        for k in ("fz", "df", "iters", "pos"):
            assert torch.equal(a[k], b[k]), (n, k)
        assert torch.equal(a["ff"][..., :3], b["ff"][..., :3]), n
        assert torch.count_nonzero(b["ff"][..., 3]).item() == 0, n


def test_graph_replay_reproduces_the_eager_run():
    cs = cases(6, 2000)
    b = batch.Batch(cs)
    b.run()
    torch.cuda.synchronize()
    eager = (b.fz.clone(), b.df.clone(), b.iters.clone())
    b.fz.fill_(float("nan"))
    b.df.fill_(float("nan"))
    b.capture()
    b.fz.fill_(float("nan"))
    b.df.fill_(float("nan"))
    b.replay()
    b.replay()
    torch.cuda.synchronize()
    assert torch.equal(b.fz, eager[0]) and torch.equal(b.df, eager[1]) and torch.equal(b.iters, eager[2])
    assert b.status() == (0, 0)


def test_bounded_wait_times_out_with_a_status():
    # relax tiles wait for one force-field tile more than exists: every wait runs out
    # after ~1000 polls; the kernel returns, the status says so, the context stays usable
    cs = cases(3, 3000)
    b = batch.Batch(cs, spin_limit=1000, wait_extra=1)
    b.run()
    st, flags = b.status()
    assert st == 5 and (flags & 2)
    ok = batch.Batch(cs)
    ok.run()
    assert ok.status() == (0, 0)
    got = ok.molecule(0)["df"].cpu().numpy()
    assert np.array_equal(got, single(cs[0])["df"])


def test_invalid_descriptor_is_skipped_and_flagged():
    cs = cases(4, 4000)
    b = batch.Batch(cs)
    raw = b.descs.cpu().numpy().copy()
    d = pp.MolDesc.from_buffer_copy(raw[ctypes.sizeof(pp.MolDesc) * 2: ctypes.sizeof(pp.MolDesc) * 3].tobytes())
    d.ff_offset = b.params.ff_capacity  # grid would run past the end of ff
    raw[ctypes.sizeof(pp.MolDesc) * 2: ctypes.sizeof(pp.MolDesc) * 3] = np.frombuffer(bytes(d), dtype=np.uint8)
    b.descs.copy_(torch.as_tensor(raw))
    b.df.fill_(7.0)
    b.run()
    st, flags = b.status()
    assert st == 4 and (flags & 1)
    for n in (0, 1, 3):
        assert np.array_equal(b.molecule(n)["df"].cpu().numpy(), single(cs[n])["df"]), n
    assert (b.molecule(2)["df"].cpu().numpy() == 7.0).all()


# Batch molecules with the extremes of the batched workload (seeds 1000 + i): the smallest grid
# (128 x 128, 13 atoms), the largest (208 x 256, 62 atoms), the least planar (2.99 A of height
# spread) and the one with the most fluorine atoms (14 of 74).
ORACLE_MOLECULES = (67, 12, 83, 104)


def test_batch_molecules_match_the_oracle(orc):
    from helpers import df_keep, ill_conditioned_within_bound, relax_compare

    cs = [case32(synth.batch_cases(1, 1000 + i)[0]) for i in ORACLE_MOLECULES]
    g0 = [c["grid"] for c in cs]
    assert min(g["nx"] * g["ny"] for g in g0) == 128 * 128 and max(g["nx"] * g["ny"] for g in g0) == 208 * 256
    assert max(float(np.ptp(c["atoms"]["z"])) for c in cs) > 2.9
    assert max(int(np.isclose(c["atoms"]["R"], 1.75).sum()) for c in cs) >= 10  # F atoms
    fire = synth.parity_fire()
    b = batch.Batch(cs, want_pos=True, fire=fire)
    b.run()
    assert b.status() == (0, 0)
    for n, c in enumerate(cs):
        got = {k: v.cpu().numpy().astype(np.float64) for k, v in b.molecule(n).items()}
        o = orc.forward(c, fire=fire)
        assert (got["iters"] < fire["max_iter"]).mean() > 0.999
        dp, dfz, keep, n_ill, n_basin = relax_compare(got, o)
        # as on the full-size flake: the far field of the wider molecules has up to ~10 % of its
        # points with lambda_min just under 0.01 eV/A^2 in the FP64 oracle itself; those are held
        # to their residual bound below, and points that settled in another basin are capped
        assert keep.mean() > 0.85, (n, n_ill, n_basin)
        assert n_basin <= 0.005 * keep.size, (n, n_basin)
        assert dp <= 1e-3, (n, dp)
        n_sel, n_ok = ill_conditioned_within_bound(got["pos"], o, fire["ftol"])
        assert n_ok == n_sel, (n, n_ok, n_sel)
        m = (keep.shape[0] - got["df"].shape[0]) // 2
        rng = o["df"].max() - o["df"].min()
        ddf = np.abs(got["df"] - o["df"])[df_keep(keep, m)].max()
        assert ddf <= 1e-3 * rng, (n, ddf, rng)


def test_every_batch_shape_gives_the_same_molecules():
    # force-field tile depth and width, relax tile width and CTA count change the schedule only:
    # every combination reproduces the default batch bit for bit, ragged scans included
    cs = cases(5, 5000)
    ref = batch.Batch(cs, want_pos=True)
    ref.run()
    assert ref.status() == (0, 0)
    want = [{k: v.clone() for k, v in ref.molecule(n).items()} for n in range(len(cs))]
    for zpt in (4, 8):
        for fw in (4, 8, 16):
            for rw in (4, 8, 16):
                b = batch.Batch(cs, want_pos=True, ff_zpt=zpt, ff_tile_w=fw, relax_tile_w=rw,
                                ctas=152 if (zpt, fw, rw) == (4, 16, 4) else 0)
                b.run()
                assert b.status() == (0, 0), (zpt, fw, rw)
                for n in range(len(cs)):
                    got = b.molecule(n)
                    for k in ("ff", "fz", "df", "iters", "pos"):
                        assert torch.equal(got[k], want[n][k]), (zpt, fw, rw, n, k)


def test_batch_tuner_picks_a_candidate_and_keeps_the_molecules():
    from paper_2401_14564_gb300 import tune

    cs = cases(4, 6000)
    b = batch.Batch(cs, want_pos=True)
    b.run()
    want = [b.molecule(n)["df"].clone() for n in range(len(cs))]
    r = tune.tune_batch(b, reps=1, factors=(1, 2))
    ch = r["choice"]
    assert ch["ff_zpt"] in (4, 8) and ch["ff_tile_w"] in (4, 8, 16) and ch["relax_tile_w"] in (4, 8, 16)
    assert (b.params.ff_zpt, b.params.ff_tile_w, b.params.relax_tile_w, b.params.ctas) == \
        (ch["ff_zpt"], ch["ff_tile_w"], ch["relax_tile_w"], ch["ctas"])
    assert r["ms"] <= r["ms_default_shapes"]
    b.run()
    for n in range(len(cs)):
        assert torch.equal(b.molecule(n)["df"], want[n])


def test_batch_shapes_are_validated():
    cs = cases(2, 7000)
    for kw in (dict(ff_tile_w=6), dict(relax_tile_w=32), dict(ff_zpt=16)):
        b = batch.Batch(cs, **kw)
        with pytest.raises(pp.PPError) as e:
            b.run()
        assert e.value.status == 1


def test_batch_from_host_memory():
    # run_host: the same atoms give the device run's images bit for bit; moved atoms give what a batch
    # built from the moved molecules (on the same grids and scans) computes
    cs = cases(4, 8000)
    b = batch.Batch(cs)
    b.run()
    want = b.df.clone()
    b.capture()
    got = b.run_host(b.pack_atoms(cs)).clone()
    assert torch.equal(got.cuda(), want)
    moved = copy.deepcopy(cs)
    for c in moved:
        c["atoms"]["x"] = (np.asarray(c["atoms"]["x"], np.float32) + np.float32(0.037)).astype(np.float64)
    ref = batch.Batch(moved)
    ref.run()
    got = b.run_host(b.pack_atoms(moved)).clone()
    assert torch.equal(got.cuda(), ref.df)
    assert b.status() == (0, 0)
