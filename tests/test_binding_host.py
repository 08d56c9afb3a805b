"""Host-side argument checks of the Python binding (no GPU).

The C ABI sees raw addresses, so the binding rejects, before any pointer
reaches the library, slices that would run past a tensor, output tensors of
the wrong size and request arrays the library would misread."""
import numpy as np
import pytest
import torch

from paper_1609_00999_gb300 import _binding, serve, synth


def _packed(lengths):
    la = np.asarray(lengths, dtype=np.int64)
    lb = la.copy()
    a_off = np.concatenate([[0], np.cumsum(la)[:-1]])
    c_off = np.concatenate([[0], np.cumsum(la + lb - 1)[:-1]])
    return a_off, la, a_off.copy(), lb, c_off, int(la.sum()), int((la + lb - 1).sum())


def test_packed_bounds_accepts_exact_fit():
    a_off, la, b_off, lb, c_off, na, nc = _packed([1, 7, 4096, 3])
    _binding._check_packed_bounds(na, a_off, la, na, b_off, lb, nc, c_off)
    _binding._check_packed_bounds(0, [], [], 0, [], [], 0, [])


@pytest.mark.parametrize("which", ["a", "b", "c"])
def test_packed_bounds_rejects_overrun(which):
    a_off, la, b_off, lb, c_off, na, nc = _packed([5, 9, 2])
    n = {"a": na, "b": na, "c": nc}
    n[which] -= 1                                   # the last product's slice now ends one word past the end
    with pytest.raises(ValueError, match="product 2: %s slice" % which):
        _binding._check_packed_bounds(n["a"], a_off, la, n["b"], b_off, lb, n["c"], c_off)


def test_packed_bounds_rejects_bad_fields():
    a_off, la, b_off, lb, c_off, na, nc = _packed([5, 9])
    with pytest.raises(ValueError, match="differ in size"):
        _binding._check_packed_bounds(na, a_off, la[:1], na, b_off, lb, nc, c_off)
    with pytest.raises(ValueError, match=">= 1"):
        _binding._check_packed_bounds(na, a_off, [5, 0], na, b_off, lb, nc, c_off)
    with pytest.raises(ValueError, match=">= 0"):
        _binding._check_packed_bounds(na, [0, -1], la, na, b_off, lb, nc, c_off)


def test_from_packed_checks_bounds_before_addresses():
    a_off, la, b_off, lb, c_off, na, nc = _packed([4, 4])
    a = torch.zeros(na, dtype=torch.int32)
    c = torch.zeros(nc - 1, dtype=torch.int32)      # one word short
    with pytest.raises(ValueError, match="c slice"):
        _binding.PolymulBatchPlan.from_packed([synth.P1] * 2, a, a_off, la, a, b_off, lb, c, c_off)


def test_polymul_many_ws_checks_out_size():
    a = torch.zeros((3, 8), dtype=torch.int32)
    out = torch.zeros((3, 14), dtype=torch.int32)   # needs 3 x 15
    with pytest.raises(ValueError, match="out must have 45 elements"):
        _binding.polymul_many_ws(synth.P1, a, a, None, out=out)


def test_request_array_checks():
    reqs = serve.make_requests([synth.P1] * 4, [8] * 4, [8] * 4, [16] * 4, [16] * 4, [16] * 4)
    _binding._check_request_array(reqs, 0, 4)
    _binding._check_request_array(reqs, 2, 2)
    with pytest.raises(ValueError):
        _binding._check_request_array(reqs, 3, 5)
    with pytest.raises(ValueError):
        _binding._check_request_array(reqs, 3, 2)
    with pytest.raises(ValueError):
        _binding._check_request_array(reqs[::2], 0, 2)
    with pytest.raises(TypeError):
        _binding._check_request_array(np.zeros(4, dtype=np.uint64), 0, 4)
    with pytest.raises(TypeError):
        _binding._check_request_array(list(reqs), 0, 4)
