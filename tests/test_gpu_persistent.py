"""The persistent frame (FEWHA_FLAG_PERSISTENT): one cooperative launch runs the whole frame
of Algorithm 1 with grid-wide waits between its stages.  Its DM commands against the FP64
oracle on warm-started sequences (graph-captured and plain stream launches), its bounded
waits (a wait that cannot end returns FEWHA_ERR_TIMEOUT and leaves the GPU usable), and the
flag combinations it refuses."""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from paper_2202_11945_gb300 import FewhaError, Reconstructor
from tests.gpu_common import TOL_FRAME, rel_l2, to_dev, to_np
from tests.test_gpu_frame import slopes

pytestmark = pytest.mark.gpu

SEQ = [("tiny_scao", 64, 6), ("tiny_scao", 32, 6), ("tiny_mcao", 64, 4), ("tiny_mcao", 32, 4),
       ("maory", 32, 4), ("maory", 64, 2), ("tiny_mcao_elongated", 32, 3), ("paper_mcao", 32, 2)]


def persistent(name, prec, graph=True, warm_residual=False):
    return Reconstructor(synth.workload_by_name(name), precision=prec, graph=graph, persistent=True,
                         warm_residual=warm_residual)


@pytest.mark.parametrize("name,prec,frames", SEQ, ids=str)
def test_sequence_matches_oracle(name, prec, frames):
    ref = O.Reconstructor(synth.workload_by_name(name))
    R = persistent(name, prec)
    assert R.frame_launches() == 1
    for t in range(frames):
        s = slopes(name, t)
        a_ref = ref.frame(s)
        a = to_np(R.reconstruct(to_dev(s, prec)))
        assert rel_l2(a, a_ref) <= TOL_FRAME[prec], (t, rel_l2(a, a_ref))
    assert not R.check_input()                  # no wait ran out, no non-finite slopes
    R.close()


@pytest.mark.parametrize("prec", [32, 64])
def test_stream_launch_and_warm_residual(prec):
    ref = O.Reconstructor(synth.workload_by_name("tiny_mcao"))
    R = persistent("tiny_mcao", prec, graph=False, warm_residual=True)
    for t in range(4):
        s = slopes("tiny_mcao", t)
        a_ref = ref.frame(s, warm_residual=True)
        a = to_np(R.reconstruct(to_dev(s, prec)))
        assert rel_l2(a, a_ref) <= TOL_FRAME[prec], (t, rel_l2(a, a_ref))
    R.close()


def test_host_buffer_frames():
    ref = O.Reconstructor(synth.workload_by_name("maory"))
    R = persistent("maory", 32)
    out = torch.empty(R.n_act, dtype=torch.float32).pin_memory()
    for t in range(2):
        s = slopes("maory", t)
        a_ref = ref.frame(s)
        R.reconstruct_host(torch.as_tensor(s, dtype=torch.float32).pin_memory(), out)
        assert rel_l2(out.double().numpy(), a_ref) <= TOL_FRAME[32], t
    R.close()


def test_a_wait_that_cannot_end_times_out_and_the_gpu_stays_usable():
    """Every wait's target is raised beyond reach (a count that no CTA completes), with a
    short poll limit: the first wait runs out, the kernel returns, and the call reports
    FEWHA_ERR_TIMEOUT.  With the limits restored, the next frames are correct."""
    name = "tiny_mcao"
    ref = O.Reconstructor(synth.workload_by_name(name))
    R = persistent(name, 32)
    R.set_wait_limit(2000, extra=1 << 20)
    s0 = slopes(name, 0)
    out = torch.empty(R.n_act, dtype=torch.float32).pin_memory()
    with pytest.raises(FewhaError) as e:
        R.reconstruct_host(torch.as_tensor(s0, dtype=torch.float32).pin_memory(), out)
    assert e.value.code == -7
    # the asynchronous entry point: the timeout shows in the status check
    R.reconstruct(to_dev(s0, 32))
    with pytest.raises(FewhaError) as e:
        R.check_input()
    assert e.value.code == -7
    R.set_wait_limit(1 << 20, extra=0)
    R.reset()
    for t in range(2):
        s = slopes(name, t)
        a = to_np(R.reconstruct(to_dev(s, 32)))
        assert rel_l2(a, ref.frame(s)) <= TOL_FRAME[32], t
    assert not R.check_input()
    R.close()


@pytest.mark.parametrize("flag", ["augmented", "closed_loop"])
def test_refused_flag_combinations(flag):
    with pytest.raises(FewhaError) as e:
        Reconstructor(synth.workload_by_name("tiny_mcao"), precision=32, persistent=True, **{flag: True})
    assert e.value.code == -1
