"""Argument marshalling of the Python binding, on the CPU: the pointers, sizes and
leading dimensions a batch hands to the C ABI address exactly the caller's
matrices, for a list and for one stacked (count, 2n, 2n) array, and malformed
batches are refused before any call."""
import ctypes

import numpy as np
import pytest

from paper_2109_04528_gb300 import binding, inputs


class HostCtx:
    flags = 0


def _view(ptr, n):
    buf = (ctypes.c_double * (2 * 4 * n * n)).from_address(int(ptr))
    return np.frombuffer(buf, dtype=np.complex128).reshape(2 * n, 2 * n)


def test_list_and_stack_address_the_matrices():
    base = inputs.lossy_squeezed(30, 5, (0.5, 1.2), 0.4).O
    rng = np.random.default_rng(1)
    mats = [inputs.submatrix(base, sorted(rng.choice(30, size=int(k), replace=False).tolist()))
            for k in rng.integers(1, 12, size=50)]
    keep, ns, lds, ptrs = binding._batch_args(HostCtx, mats)
    assert ns.dtype == np.int32 and lds.dtype == np.int32 and ptrs.dtype == np.uint64
    for O, n, ld, p in zip(mats, ns, lds, ptrs):
        assert n == O.shape[0] // 2 and ld == O.shape[0]
        assert np.array_equal(_view(p, n), O)
    same = [m for m in mats if m.shape[0] == mats[0].shape[0]]
    stack = np.stack(same)
    keep, ns, lds, ptrs = binding._batch_args(HostCtx, stack)
    for i, O in enumerate(same):
        assert ns[i] == O.shape[0] // 2 and lds[i] == O.shape[0]
        assert np.array_equal(_view(ptrs[i], ns[i]), O)
    # a non-contiguous stack is copied once, still addressed right
    keep, ns, lds, ptrs = binding._batch_args(HostCtx, np.stack([x for m in same for x in (m, m)])[::2])
    assert np.array_equal(_view(ptrs[1], ns[1]), same[1])


def test_mixed_and_converted_inputs_take_the_general_path():
    a = np.eye(4)  # float: converted to complex128 and kept alive
    b = np.asfortranarray(inputs.lossy_squeezed(3, 2).O)  # not C-contiguous
    keep, ns, lds, ptrs = binding._batch_args(HostCtx, [a, b])
    assert list(ns) == [2, 3] and list(lds) == [4, 6]
    assert np.array_equal(_view(ptrs[0], 2), a.astype(np.complex128))
    assert np.array_equal(_view(ptrs[1], 3), np.ascontiguousarray(b))


@pytest.mark.parametrize("bad", [[np.zeros((3, 3), complex)], [np.zeros((4, 6), complex)],
                                 np.zeros((2, 4, 6), complex), np.zeros((2, 3, 3), complex)])
def test_malformed_batches_are_refused(bad):
    with pytest.raises(binding.TorError):
        binding._batch_args(HostCtx, bad)


def test_result_records_have_the_c_layout():
    assert binding.RESULT_DTYPE.itemsize == ctypes.sizeof(binding.tor_result)
    for name, _ in binding.tor_result._fields_:
        assert binding.RESULT_DTYPE.fields[name][1] == getattr(binding.tor_result, name).offset
    rec = np.zeros(2, dtype=binding.RESULT_DTYPE)
    rec[1] = (1.5, 2.0 ** -60, 3.0, 1e-9, 7, 0, 1, 0)
    r = binding._results(rec)[1]
    assert (r.hi, r.lo, r.abs_sum, r.err_est, r.n, r.status, r.path) == (1.5, 2.0 ** -60, 3.0, 1e-9, 7, 0, 1)
