"""Device-allocation failures and the instance's device footprint.

The library's allocation wrapper can be told to fail the n-th next allocation
(fewha_test_fail_alloc), as if the device were out of memory.  fewha_create and the
allocations made on first use of an option must then return FEWHA_ERR_OOM, release what
they had allocated, and leave the instance (or the process) usable."""
import numpy as np
import pytest
import torch

import synth
from paper_2202_11945_gb300 import FewhaError, Reconstructor, lib
from tests.gpu_common import to_dev, to_np

pytestmark = pytest.mark.gpu

OOM = -3


def fail_after(n):
    lib().fewha_test_fail_alloc(int(n))


def free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


@pytest.mark.parametrize("prec", [32, 64])
def test_create_fails_cleanly_at_every_allocation(prec):
    wl = synth.maory()
    free0 = free_bytes()
    failures = 0
    for after in range(0, 400):
        fail_after(after)
        try:
            R = Reconstructor(wl, precision=prec)
        except FewhaError as e:
            assert e.code == OOM, e
            failures += 1
            continue
        finally:
            fail_after(-1)
        # the first `after` that lets the creation through: every allocation point was hit
        assert R.device_bytes() > 0
        R.close()
        break
    assert failures >= 20, failures
    # nothing was kept by the failed creations (the driver's granularity is 2 MiB pages)
    assert abs(free_bytes() - free0) < (32 << 20), (free0, free_bytes())


def test_allocations_on_first_use_fail_cleanly():
    wl = synth.tiny_mcao()
    s = to_dev(synth.simulate_slopes(wl, 0), 32)
    # augmented PCG: the direction sets are allocated by the first frame
    R = Reconstructor(wl, precision=32, augmented=True)
    before = R.device_bytes()
    fail_after(0)
    with pytest.raises(FewhaError) as e:
        R.reconstruct(s)
    fail_after(-1)
    assert e.value.code == OOM
    assert R.device_bytes() == before
    a = to_np(R.reconstruct(s))
    assert np.all(np.isfinite(a)) and R.device_bytes() > before
    R.close()
    # the double-precision copy of a single-precision instance's converged solve
    R = Reconstructor(wl, precision=32)
    before = R.device_bytes()
    fail_after(0)
    with pytest.raises(FewhaError) as e:
        R.reconstruct_converged(s, tol=1e-8, max_iters=20000)
    fail_after(-1)
    assert e.value.code == OOM and R.device_bytes() == before
    dm, it, rel = R.reconstruct_converged(s, tol=1e-8, max_iters=20000)
    assert rel <= 1e-8 and R.device_bytes() > before
    R.close()
    # the reverse pass's record of the frame
    R = Reconstructor(wl, precision=64, graph=False)
    c0 = torch.zeros(R.n_coeffs, dtype=torch.float64, device="cuda")
    g = torch.ones(R.n_act, dtype=torch.float64, device="cuda")
    s64 = s.double()
    before = R.device_bytes()
    fail_after(0)
    with pytest.raises(FewhaError) as e:
        R.frame_vjp(s64, c0, g)
    fail_after(-1)
    assert e.value.code == OOM and R.device_bytes() == before
    a, gs = R.frame_vjp(s64, c0, g)
    assert np.all(np.isfinite(to_np(gs)))
    R.close()


def test_footprint_of_the_maory_instance():
    """The instance's own accounting against the device's free memory, and the scale the
    paper compares (Sec. 4.3: 16 MB for FEWHA against 53 GB for a matrix-vector method)."""
    wl = synth.maory()
    for prec, hi in ((32, 40 << 20), (64, 80 << 20)):
        free0 = free_bytes()
        R = Reconstructor(wl, precision=prec)
        held = R.device_bytes()
        used = free0 - free_bytes()
        assert 0 < held <= hi, held
        # the device's free memory moves by whole pages, and small allocations come from pools
        # the driver reserves ahead: the drop only has to be of the same order
        assert used < held + (64 << 20), (used, held)
        R.close()
