"""Failure detection without a GPU fault.

* bse_sync's host-side deadline: a host function on the context's stream keeps it busy
  (bse_selftest_delay), so a sync with a shorter limit returns BSE_ETIMEOUT while the work
  keeps running, and a later sync waits for it and succeeds.
* The bounded device wait of the tensor-core and matvec pipelines: bse_selftest_wait waits on
  a barrier nothing completes, gives up after its cycle limit and sets the error word; the
  next bse_sync returns BSE_ETIMEOUT and the context stays usable (an assembly that follows
  still matches the oracle).
* A device-side check: a zero energy denominator in the dipole vector gives BSE_EDEVICE."""
import time

import numpy as np
import pytest

import oracle as O
from synth import config_spec, make_inputs

from helpers import gpu_hamiltonian, to_dev

pytestmark = pytest.mark.gpu


def _ctx():
    from paper_2607_05853_b300.api import BSE
    inp = make_inputs(config_spec(0))
    return inp, BSE.from_inputs(inp, precision="bf16x3")


def test_sync_deadline_on_a_busy_stream():
    from paper_2607_05853_b300 import _lib
    inp, b = _ctx()
    b.selftest_delay(1500)
    t0 = time.perf_counter()
    with pytest.raises(_lib.BseError) as e:
        b.sync(timeout_ms=100)
    waited = time.perf_counter() - t0
    assert e.value.status == _lib.BSE_ETIMEOUT
    assert 0.09 <= waited <= 1.0
    b.sync(timeout_ms=10_000)          # the delay ends; nothing was lost
    b.sync(timeout_ms=0)               # an idle stream passes a zero limit
    b.close()


def test_bounded_device_wait_reports_timeout_and_context_survives():
    from paper_2607_05853_b300 import _lib
    inp, b = _ctx()
    b.selftest_wait(200_000_000)       # ~0.1 s at 2 GHz
    with pytest.raises(_lib.BseError) as e:
        b.sync(timeout_ms=20_000)
    assert e.value.status == _lib.BSE_ETIMEOUT
    assert "bounded device wait" in str(e.value)
    b.sync(timeout_ms=1000)            # the error word was read and cleared
    d = to_dev(inp)
    b.interp_W(d["W_R"], d["V0"])
    b.project_pairs(d["C_R"], d["c_k"], d["e_qp"])
    H = b.assemble()
    b.sync()
    ref = O.BSEOracle(inp).hamiltonian()
    assert np.abs(H.cpu().numpy() - ref).max() <= 1e-5 * np.abs(ref).max()
    b.close()


def test_zero_denominator_is_a_device_error():
    import torch
    from paper_2607_05853_b300 import _lib
    inp, b = _ctx()
    d = to_dev(inp)
    e_ks = d["e_ks"].clone()
    e_ks[3, b.nv] = e_ks[3, 0]          # E_c = E_v at one k
    b.dipole_vector(d["vel"], e_ks)
    with pytest.raises(_lib.BseError) as e:
        b.sync()
    assert e.value.status == _lib.BSE_EDEVICE
    b.sync()
    b.close()
