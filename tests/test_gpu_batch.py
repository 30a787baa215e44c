"""Batched frames of uneven instances: one launch per step over all instances' work items.

The batched kernels run the single-instance kernel bodies on (instance, unit) items, so a
batched frame must give each instance the same commands, bit for bit, as its own frame
(for the vector kernel's default partition); other partitions of the vector kernel change
only the summation order of r.z and stay within the frame tolerance of the oracle."""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from tests.gpu_common import TOL_FRAME, rel_l2, to_dev, to_np

pytestmark = pytest.mark.gpu

_cache = {}


def instances():
    """Small test batch: the test workloads plus the first instances of the uneven set."""
    if "wl" not in _cache:
        wls = [synth.tiny_scao(), synth.tiny_mcao()] + synth.batched_instances(10)
        seqs = []
        for wl in wls:
            atm = synth.TruthAtmosphere(wl["truth"])
            seqs.append([synth.simulate_slopes(wl, t, atm=atm) for t in range(3)])
        _cache["wl"] = (wls, seqs)
    return _cache["wl"]


def make(wls, precision=32, warm_residual=False):
    from paper_2202_11945_gb300 import Reconstructor
    return [Reconstructor(wl, precision=precision, warm_residual=warm_residual) for wl in wls]


def frames_single(recons, seqs, precision):
    out = []
    for R, seq in zip(recons, seqs):
        out.append([to_np(R.reconstruct(to_dev(s, precision))) for s in seq])
    return out


def frames_batched(B, recons, seqs, precision):
    out = [[] for _ in recons]
    for t in range(len(seqs[0])):
        dms = B.reconstruct([to_dev(seq[t], precision) for seq in seqs])
        for i, d in enumerate(dms):
            out[i].append(to_np(d))
    return out


# the projection kernels' CTA size and tap unroll change which thread computes an element,
# not its arithmetic: those shapes stay bit-identical to the single-instance frames
@pytest.mark.parametrize("cfg", [dict(order=0, groups=1, vec_passes=1),
                                 dict(order=1, groups=1, vec_passes=1),
                                 dict(order=1, groups=3, vec_passes=1),
                                 dict(order=0, groups=8, vec_passes=1),
                                 dict(order=0, groups=2, vec_passes=1, pair_threads=256, proj_taps=8)], ids=str)
def test_batched_frames_equal_single_frames_bitwise(cfg):
    from paper_2202_11945_gb300 import Batch
    wls, seqs = instances()
    ref = frames_single(make(wls), seqs, 32)
    recons = make(wls)
    B = Batch(recons)
    B.config = cfg
    got = frames_batched(B, recons, seqs, 32)
    for i in range(len(wls)):
        for t in range(len(seqs[0])):
            assert np.array_equal(got[i][t], ref[i][t]), (wls[i]["name"], t, cfg)
    B.close()


def test_four_tap_adjoint_projection_and_small_ctas_are_bitwise():
    """Where every member touches at most 4 aperture rows per layer row (the 8 m
    single-conjugate geometry), the 4-tap adjoint projection is available and, like the
    half-size projection CTAs, leaves the frames bit-identical; a 4-tap request on a batch
    that needs more taps is refused."""
    from paper_2202_11945_gb300 import Batch, FewhaError
    wls, seqs = instances()
    sub = [wls[0], synth.tiny_scao()]
    sq = [seqs[0], seqs[0]]
    ref = frames_single(make(sub), sq, 32)
    recons = make(sub)
    B = Batch(recons)
    B.config = dict(order=0, groups=1, vec_passes=1, pair_threads=256, proj_taps=4)
    got = frames_batched(B, recons, sq, 32)
    for i in range(2):
        for t in range(len(sq[0])):
            assert np.array_equal(got[i][t], ref[i][t]), (i, t)
    B.close()
    B = Batch(make(wls))
    with pytest.raises(FewhaError):
        B.config = dict(order=0, groups=1, vec_passes=1, proj_taps=4)
    B.close()


def test_vector_partitions_stay_within_tolerance_of_the_oracle():
    from paper_2202_11945_gb300 import Batch
    wls, seqs = instances()
    small = [0, 1, 4, 8]                      # instances the oracle runs in seconds
    sub = [wls[i] for i in small]
    recons = make(sub)
    B = Batch(recons)
    B.config = dict(order=1, groups=2, vec_passes=4, vec_threads=512, pair_threads=256)
    assert B.config["vec_threads"] == 512 and B.config["pair_threads"] == 256
    got = frames_batched(B, recons, [seqs[i] for i in small], 32)
    for k, i in enumerate(small):
        ref = O.Reconstructor(wls[i])
        for t in range(len(seqs[i])):
            a = ref.frame(seqs[i][t])
            assert rel_l2(got[k][t], a) <= TOL_FRAME[32], (wls[i]["name"], t)
    B.close()


def test_fp64_batch_matches_oracle():
    from paper_2202_11945_gb300 import Batch
    wls, seqs = instances()
    small = [0, 1, 2]
    recons = make([wls[i] for i in small], precision=64)
    B = Batch(recons)
    got = frames_batched(B, recons, [seqs[i] for i in small], 64)
    for k, i in enumerate(small):
        ref = O.Reconstructor(wls[i])
        for t in range(len(seqs[i])):
            assert rel_l2(got[k][t], ref.frame(seqs[i][t])) <= TOL_FRAME[64], (wls[i]["name"], t)
    B.close()


def test_warm_residual_batch_equals_single():
    from paper_2202_11945_gb300 import Batch
    wls, seqs = instances()
    sub = wls[:4]
    ref = frames_single(make(sub, warm_residual=True), seqs[:4], 32)
    recons = make(sub, warm_residual=True)
    B = Batch(recons)
    got = frames_batched(B, recons, seqs[:4], 32)
    for i in range(len(sub)):
        for t in range(len(seqs[0])):
            assert np.array_equal(got[i][t], ref[i][t]), (i, t)
    B.close()


def test_autotune_keeps_state_and_is_remembered():
    from paper_2202_11945_gb300 import Batch
    wls, seqs = instances()
    sub = wls[2:8]
    ref = frames_single(make(sub), seqs[2:8], 32)
    recons = make(sub)
    B = Batch(recons)
    cfg, us = B.autotune([to_dev(seq[0], 32) for seq in seqs[2:8]], reps=3)
    assert us > 0 and 1 <= cfg["groups"] <= 8 and cfg["order"] in (0, 1)
    B.config = dict(cfg, vec_passes=1)
    got = frames_batched(B, recons, seqs[2:8], 32)
    for i in range(len(sub)):
        for t in range(len(seqs[0])):
            assert np.array_equal(got[i][t], ref[i][t]), (i, t)
    B2 = Batch(make(sub))                     # same shapes: starts from the tuned config
    assert B2.config == cfg
    B.close()
    B2.close()


def test_convenience_entry_point_matches_batch_object():
    from paper_2202_11945_gb300 import Batch, reconstruct_batched
    wls, seqs = instances()
    sub = wls[:5]
    A = make(sub)
    Bh = make(sub)
    B = Batch(Bh)
    for t in range(2):
        s = [to_dev(seq[t], 32) for seq in seqs[:5]]
        a = reconstruct_batched(A, s)
        b = B.reconstruct(s)
        for x, y in zip(a, b):
            assert np.array_equal(to_np(x), to_np(y))
    B.close()


def test_batch_argument_errors():
    from paper_2202_11945_gb300 import Batch, FewhaError
    wls, seqs = instances()
    R = make(wls[:2])
    with pytest.raises(FewhaError):
        Batch([R[0], R[0]])                          # a handle twice
    R64 = make(wls[:1], precision=64)
    with pytest.raises(FewhaError):
        Batch([R[0], R64[0]])                        # mixed precision
    R4 = make(wls[:2])
    R4[1].update_params(iters=3)
    B = Batch(R4)
    with pytest.raises(FewhaError):
        B.reconstruct([to_dev(seqs[0][0], 32), to_dev(seqs[1][0], 32)])   # different iterations
    B.close()
    Rd = make(wls[:2])
    B = Batch(Rd)
    s = [to_dev(seqs[0][0], 32), to_dev(seqs[1][0], 32)]
    B.reconstruct(s)
    Rd[1].close()                                    # a member goes away
    with pytest.raises(FewhaError):
        B.reconstruct(s)
    B.close()
