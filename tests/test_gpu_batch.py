"""Batched ensembles: many independent systems of uneven size (channels and sphere-pack
pores) advanced together, one launch per phase over all of them, replayed from CUDA
graphs.  Each system must follow bit for bit the trajectory it follows alone, and one
batched step must match the oracle like a single system's step does."""
import numpy as np
import pytest

import oracle
from paper_1807_09896_gb300 import dpd, inputs
from parity_helpers import compare_one_step, first_newton3_variant, gpu_state, make_system, params_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1807_09896_gb300 import _build

    _build.build()


def _small_ensemble(n=6, seed=3):
    return inputs.ensemble(n, seed=seed, min_fluid=400, max_fluid=6000, edge=(6, 12), gap=(4, 10))


def _systems(ws, **opts):
    out = []
    for k, w in enumerate(ws):
        p = params_for(w, g=(0.02, 0.0, 0.0), seed=100 + k, sys=k)
        out.append((make_system(w, p, **opts), p))
    return out


def _batch_state(b, k):
    pos4, vel4, f4, ids, types = dpd.dpd_batch_get_state(b.hb, k)
    assert np.array_equal(ids, np.arange(len(ids)))
    return pos4[:, :3].copy(), vel4[:, :3].copy(), f4[:, :3].copy(), types


def test_batched_systems_follow_their_solo_trajectories_bitwise():
    ws = _small_ensemble()
    alone = _systems(ws)
    for s, _ in alone:
        s.step(33)
    members = _systems(ws)
    b = dpd.Batch([s for s, _ in members], graph_steps=10)
    b.step(33)
    for k, (s, _) in enumerate(alone):
        for x, y in zip(gpu_state(s), _batch_state(b, k)):
            np.testing.assert_array_equal(x, y)
        np.testing.assert_array_equal(s.stats()[5:], dpd.dpd_batch_get_stats(b.hb, k)[5:])
    b.close()


def test_batch_autotune_and_launch_shapes_keep_trajectories():
    """Tuning a batch leaves its state as it was; with the chosen shape the members
    still follow their solo trajectories bit for bit."""
    ws = _small_ensemble(4, seed=7)
    members = _systems(ws)
    b = dpd.Batch([s for s, _ in members])
    chosen, ms = dpd.dpd_batch_autotune(b.hb, 2)
    assert int(dpd.dpd_batch_get_stats(b.hb, 0)[7]) == 0
    b.step(12)
    alone = _systems(ws)  # loaded (f(0)) with the default shape, as the members were
    for s, _ in alone:
        s.set_option("force_variant", chosen)
        s.step(12)
    for k, (s, _) in enumerate(alone):
        for x, y in zip(gpu_state(s), _batch_state(b, k)):
            np.testing.assert_array_equal(x, y)
    assert 0 <= chosen < len(ms)
    b.close()


def test_newton3_batch_members_follow_their_solo_trajectories_bitwise():
    """Fixed-point sums do not depend on the order of the atomics, so a member of a
    batch using the Newton's-third-law force shapes matches its solo run bit for bit."""
    ws = _small_ensemble(5, seed=9)
    probe = _systems(ws[:1])[0][0]
    v3 = first_newton3_variant(probe)
    alone = _systems(ws)  # loaded (f(0)) with the default shape, as the members were
    for s, _ in alone:
        s.set_option("force_variant", v3)
        s.step(17)
    members = _systems(ws)
    b = dpd.Batch([s for s, _ in members], force_variant=v3, graph_steps=8)
    b.step(17)
    for k, (s, _) in enumerate(alone):
        for x, y in zip(gpu_state(s), _batch_state(b, k)):
            np.testing.assert_array_equal(x, y)
    b.close()


class _Member:
    """One system of a batch, seen through the System interface the parity helper uses."""

    def __init__(self, b, k):
        self.b, self.k = b, k

    def state(self):
        return dpd.dpd_batch_get_state(self.b.hb, self.k)

    def stats(self):
        return dpd.dpd_batch_get_stats(self.b.hb, self.k)

    def get_option(self, key):
        assert key == "step"
        return self.stats()[7]

    def step(self, n=1):
        self.b.step(n)


def test_a_batched_step_matches_the_oracle_for_every_member():
    ws = _small_ensemble(4, seed=11)
    members = _systems(ws)
    b = dpd.Batch([s for s, _ in members])
    b.step(6)
    for k, (w, (s, p)) in enumerate(zip(ws, members)):
        compare_one_step(_Member(b, k), w, p, oracle.Field(w.phi, w.h), label=f"batch member {k}")
    b.close()


def test_batch_rejects_unloaded_or_repeated_systems():
    w = inputs.channel(5.0, 5.0, 4.0, seed=1)
    p = params_for(w)
    s_unloaded = make_system(w, p, load=False)
    s_ok = make_system(w, p)
    with pytest.raises(dpd.DPDError) as e:
        dpd.Batch([s_ok, s_unloaded])
    assert e.value.code == dpd.DPD_ESTATE
    with pytest.raises(dpd.DPDError) as e:
        dpd.Batch([s_ok, s_ok])
    assert e.value.code == dpd.DPD_EINVAL


def test_full_size_ensemble_matches_its_solo_runs_and_the_oracle():
    """The benchmark's 64-system ensemble at full size (alternating channels and
    sphere-pack pores of 2k-60k fluid particles, about 1.78 M in all, body force 0.01 in
    the channels and 0.005 in the pores), autotuned as the benchmark does: after 20
    steps replayed from the batch's graph every member equals its solo run bit for bit,
    and one further batched step matches the oracle member by member."""
    ws = inputs.ensemble(64, seed=0)
    ps = [params_for(w, g=(0.01 if w.gap else 0.005, 0.0, 0.0), seed=k, sys=k) for k, w in enumerate(ws)]
    members = [make_system(w, p) for w, p in zip(ws, ps)]
    b = dpd.Batch(members, graph_steps=20)
    chosen, _ = dpd.dpd_batch_autotune(b.hb, 2)
    b.step(20)
    for k, (w, p) in enumerate(zip(ws, ps)):
        s = make_system(w, p)  # loaded (f(0)) with the default shape, as the member was
        s.set_option("force_variant", chosen)
        s.step(20)
        for x, y in zip(gpu_state(s), _batch_state(b, k)):
            np.testing.assert_array_equal(x, y, err_msg=f"member {k}")
        s.close()
    for k, (w, p) in enumerate(zip(ws, ps)):
        compare_one_step(_Member(b, k), w, p, oracle.Field(w.phi, w.h), label=f"ensemble member {k}")
    b.close()
    for s in members:
        s.close()
