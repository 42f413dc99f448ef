"""tor_eval_noalloc: the entry point for callers that cannot allocate memory
while they run (pre-reserved device pools, latency-critical loops where an
allocation would synchronise the device, plugins restricted to start-up
allocation).  It keeps every intermediate buffer in a static device array, so
this test checks that it gives the same answers as tor_eval and as the CPU
oracle, on two calls in a row that share that array, and that it refuses sizes
it has no room for.

The test file is named so that pytest collects it last; it builds the library
itself and passes alone in a fresh process as well as after the other tests.
"""
import ctypes

import numpy as np
import pytest

from paper_2109_04528_gb300 import binding, build, inputs

pytestmark = pytest.mark.gpu
TOL = 1e-10


def _call(lib, torch, O_dev, n, stream):
    out = torch.zeros(ctypes.sizeof(binding.tor_result), dtype=torch.uint8, device=O_dev.device)
    st = lib.tor_eval_noalloc(O_dev.device.index, n, ctypes.c_void_p(O_dev.data_ptr()), O_dev.stride(0),
                              binding.TOR_LAYOUT_BLOCK, ctypes.c_void_p(stream), ctypes.c_void_p(out.data_ptr()))
    return st, out


def _read(torch, out):
    torch.cuda.synchronize()
    return binding.tor_result.from_buffer_copy(bytes(out.cpu().numpy()))


def test_noalloc_matches_tor_eval_twice_in_a_row(oracle_mod):
    torch = pytest.importorskip("torch")
    build.build()
    lib = binding.load_library()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev).cuda_stream
    cases = [inputs.lossy_squeezed(16, 4242, (0.3, 0.8), (0.3, 0.7)),  # shared-prefix path (p >= 5)
             inputs.lossy_squeezed(9, 4243, (0.5, 1.2), 0.4)]          # lane-built roots (p < 5)
    with binding.Context(device=0) as ctx:
        for inst in cases:
            ref = binding.tor_eval(ctx, inst.O)
            exact = oracle_mod.tor_brute(inst.O)  # binary128, every subset (Eq. tor)
            O_dev = torch.from_numpy(inst.O).to(dev)
            for _ in range(2):  # the second call reuses what the first left in the array
                st, out = _call(lib, torch, O_dev, inst.n, stream)
                assert st == binding.TOR_OK
                r = _read(torch, out)
                assert r.status == binding.TOR_OK and r.n == inst.n
                assert abs((r.hi - ref.hi) + (r.lo - ref.lo)) <= TOL * ref.abs_sum
                assert abs(r.abs_sum - ref.abs_sum) <= 1e-12 * ref.abs_sum
                assert abs((r.hi - exact.hi) + (r.lo - exact.lo)) <= TOL * exact.abs_sum
                assert abs(r.abs_sum - exact.abs_sum) <= 1e-12 * exact.abs_sum


def test_noalloc_rejects_what_does_not_fit():
    torch = pytest.importorskip("torch")
    build.build()
    lib = binding.load_library()
    dev = torch.device("cuda", 0)
    big = torch.zeros((2 * 17, 2 * 17), dtype=torch.complex128, device=dev)
    st, _ = _call(lib, torch, big, 17, torch.cuda.current_stream(dev).cuda_stream)
    assert st == binding.TOR_ETOOBIG
    # the entry point is still usable afterwards, and reports per-matrix errors in out->status
    not_pd = torch.from_numpy(2 * np.eye(8, dtype=np.complex128)).to(dev)
    st, out = _call(lib, torch, not_pd, 4, torch.cuda.current_stream(dev).cuda_stream)
    assert st == binding.TOR_OK and _read(torch, out).status == binding.TOR_ENOTPD
