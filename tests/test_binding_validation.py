"""Host-side checks of the binding's argument validation (no GPU needed).

The local-matvec wrappers must refuse operands whose dtype, device or shape
disagree before anything reaches the library: a float32 PhiL beside float64
x would make the kernels read twice the buffer's bytes, and a short y would
be written past its end.  Stand-in tensor objects carry only what the
validator reads (no data, no device memory)."""
import numpy as np
import pytest
import torch

from paper_1811_06797_gb300 import iga


class FakeCuda:
    def __init__(self, shape, dtype=torch.float64, device="cuda:0", contiguous=True, ptr=None):
        self.shape = tuple(shape)
        self.dtype = dtype
        self.device = torch.device(device)
        self.is_cuda = True
        self._contig = contiguous
        self._ptr = ptr if ptr is not None else id(self)

    def is_contiguous(self):
        return self._contig

    def dim(self):
        return len(self.shape)

    def data_ptr(self):
        return self._ptr


def operands(**over):
    r0, n, r1, R0, R1, p, nvec = 3, 7, 4, 2, 5, 2, 2
    ops = {"PhiL": FakeCuda((R0, r0, r0)), "bands": FakeCuda((R0, R1, n, 2 * p + 1)),
           "PhiR": FakeCuda((R1, r1, r1)), "x": FakeCuda((nvec, r0, n, r1)),
           "y": FakeCuda((nvec, r0, n, r1))}
    ops.update(over)
    return ops


def check(**over):
    o = operands(**{k: v for k, v in over.items() if k != "bandmask"})
    return iga._local_matvec_args(o["PhiL"], o["bands"], o["PhiR"], o["x"], o["y"],
                                  over.get("bandmask"))


def test_valid_operands_pass():
    sizes, mask, keep = check()
    assert sizes == (3, 7, 4, 2, 5, 2, 2) and mask is None
    sizes, mask, keep = check(bandmask=np.ones((2, 5), bool))
    assert mask is not None and keep.size == 10


@pytest.mark.parametrize("bad", [
    {"PhiL": FakeCuda((2, 3, 3), dtype=torch.float32)},        # mixed precision
    {"y": FakeCuda((2, 3, 7, 4), dtype=torch.float32)},
    {"bands": FakeCuda((2, 5, 7, 5), device="cuda:1")},        # another device
    {"x": FakeCuda((2, 3, 7, 4), contiguous=False)},
    {"y": FakeCuda((2, 3, 6, 4))},                             # short output
    {"bands": FakeCuda((2, 5, 7, 4))},                         # even band width
    {"bands": FakeCuda((2, 4, 7, 5))},                         # R1 disagrees with PhiR
    {"PhiL": FakeCuda((2, 3, 4))},                             # not square
    {"x": FakeCuda((2, 4, 7, 4))},                             # r0 disagrees with PhiL
    {"bandmask": np.ones(9, bool)},                            # mask of the wrong size
])
def test_mismatched_operands_raise_before_any_launch(bad):
    with pytest.raises(iga.IgaError) as e:
        check(**bad)
    assert e.value.status == 1


def test_aliased_input_and_output_raise():
    x = FakeCuda((2, 3, 7, 4), ptr=1234)
    y = FakeCuda((2, 3, 7, 4), ptr=1234)
    with pytest.raises(iga.IgaError):
        check(x=x, y=y)


def test_cpu_tensor_raises():
    with pytest.raises(iga.IgaError):
        check(PhiR=torch.zeros((5, 4, 4), dtype=torch.float64))
