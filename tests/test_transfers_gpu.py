"""Host transfers through the C ABI: the batched calls (ocn_set_fields / ocn_get_fields) against
the single-field calls and the device path, bit for bit, on a stepped FP32 LES state with two
tracers (whose full values the calls form from the stored anomalies and reference profiles), and
the order of transfers against the model stream when two models share the GPU."""
import numpy as np
import pytest

from paper_2502_14148_gb300 import inputs

pytestmark = pytest.mark.gpu


def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_14148_gb300 import ocn
    return torch, ocn


def _host(torch, st, names):
    return {n: torch.from_numpy(np.ascontiguousarray(st[n], dtype=np.float32)).pin_memory() for n in names}


def test_batched_transfers_match_single_field_calls():
    torch, ocn = _gpu()
    p = inputs.config("les_512", Nx=48, Ny=24, Nz=18)
    st = inputs.initial_state(p)
    a, b = ocn.Model(p), ocn.Model(p)
    names = ["u", "v", "w"] + a.tracers
    host = _host(torch, st, names)
    a.set_host_many(host)                       # batched
    for n in names:                             # one field per call
        b.set_host(n, host[n])
    for m in (a, b):
        m.project()
        m.time_step(p["dt"], 2)
    out_a = {n: torch.empty(a.shape(n), dtype=torch.float32).pin_memory() for n in names}
    out_b = {n: torch.empty(b.shape(n), dtype=torch.float32).pin_memory() for n in names}
    a.get_host_many(out_a)
    for n in names:
        b.get_host(n, out_b[n])
    for n in names:
        dev = a.get_numpy(n)
        assert np.array_equal(out_a[n].numpy(), dev), n          # batched get = device path
        assert np.array_equal(out_a[n].numpy(), out_b[n].numpy()), n   # batched = single-field calls
    # a second get after one more step: the work array of the batched get is the state buffer the
    # step does not read, so stepping on from the current state is unaffected by the first get
    for m in (a, b):
        m.time_step(p["dt"], 1)
    a.get_host_many(out_a)
    for n in names:
        b.get_host(n, out_b[n])
        assert np.array_equal(out_a[n].numpy(), out_b[n].numpy()), n


@pytest.mark.parametrize("wait", [True, False])
def test_transfers_ordered_against_steps_of_two_models(wait):
    """Two models alternating as in the end-to-end benchmark: step i's fields are set and its step
    launched before step i-1's fields are read back, with the host waiting for each transfer or
    (OCN_HOST_ASYNC) only once, at the end; every readout equals that of a model stepped on its
    own."""
    torch, ocn = _gpu()
    p = inputs.config("les_512", Nx=32, Ny=32, Nz=16)
    st = inputs.initial_state(p)
    ref = ocn.Model(p)
    names = ["u", "v", "w"] + ref.tracers
    host = _host(torch, st, names)
    ref.set_host_many(host)
    ref.time_step(p["dt"], 1)
    want = {n: ref.get_numpy(n) for n in names}
    pair = (ocn.Model(p), ocn.Model(p))
    got = []
    pair[0].set_host_many(host, wait)
    pair[0].time_step(p["dt"], 1)
    for i in range(1, 5):
        x, y = pair[i % 2], pair[(i - 1) % 2]
        x.set_host_many(host, wait)
        x.time_step(p["dt"], 1)
        out = {n: torch.empty(ref.shape(n), dtype=torch.float32).pin_memory() for n in names}
        y.get_host_many(out, wait)
        got.append(out)
    for m in pair:
        m.wait_transfers()
    for i, out in enumerate(got):
        for n in names:
            assert np.array_equal(out[n].numpy(), want[n]), (i, n)
