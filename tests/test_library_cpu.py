"""CPU-side checks of the C ABI library: it builds for sm_103a, loads, exports
every function include/akmc.h declares, and validates inputs on the host
(akmc_workspace_bytes makes no device call)."""
import copy
import ctypes
import os
import re

import numpy as np

import pytest

import synth
from paper_2604_24091_gb300 import akmc as A
from paper_2604_24091_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return A.load_library()


def test_exports_every_declared_symbol(lib):
    hdr = open(os.path.join(ROOT, "include", "akmc.h")).read()
    names = set(re.findall(r"\b(akmc_[a-z_0-9]+)\s*\(", hdr))
    assert len(names) >= 12
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_workspace_bytes_sizes_and_validation(lib, model):
    d = synth.config_batched_eam(4)
    n4 = A.workspace_bytes(d, model)
    n8 = A.workspace_bytes(synth.config_batched_eam(8), model)
    # species (64 KiB) + density (256 KiB) per 32^3-cell voxel at least
    assert n8 - n4 >= 4 * (65536 + 4 * 65536)
    assert A.workspace_bytes(synth.config_plain_pair(), model) < n4
    bad = [synth.VoxelDesc(2, 1, (0, 0, 0), 563.0, 0)]                      # L too small
    with pytest.raises(A.AkmcError):
        A.workspace_bytes(bad, model)
    with pytest.raises(A.AkmcError):
        A.workspace_bytes([synth.VoxelDesc(4, 0, (0, 0, 0), 563.0, 0)], model)    # no vacancy
    A.workspace_bytes([synth.VoxelDesc(16, 256, (0, 0, 0), 563.0, 0)], model)  # the most vacancies allowed
    with pytest.raises(A.AkmcError):
        A.workspace_bytes([synth.VoxelDesc(16, 257, (0, 0, 0), 563.0, 0)], model)  # one more
    with pytest.raises(A.AkmcError):
        A.workspace_bytes([synth.VoxelDesc(4, 1, (0.6, 0.6, 0), 563.0, 0)], model)  # over-full
    m = copy.deepcopy(model)
    m.eps1 = m.eps1 + 1e-9                                                       # not dyadic
    with pytest.raises(A.AkmcError):
        A.workspace_bytes(synth.config_plain_pair(), m)
    m = copy.deepcopy(model)
    m.rho_h = 0.003                                                              # not a power of two
    with pytest.raises(A.AkmcError):
        A.workspace_bytes(synth.config_batched_eam(1), m)
    assert "power of two" in A.last_error()


def test_oracle_and_library_share_no_source():
    csrc = os.path.join(ROOT, "paper_2604_24091_gb300", "csrc")
    for f in os.listdir(csrc):
        text = open(os.path.join(csrc, f)).read()
        assert "oracle" not in text.lower() or f.endswith(".md")
    for f in ("akmc_oracle.cpp", "akmc_oracle.h", "__init__.py"):
        text = open(os.path.join(ROOT, "oracle", f)).read()
        assert "akmc_device" not in text and "paper_2604_24091_gb300" not in text


def test_select_plan_sizing_and_validation(lib):
    # host-side planning of the global selection (no device needed): parts of
    # up to 8192 logits per segment, invalid offsets rejected with 0 bytes
    L = A.load_library()

    def nbytes(off):
        a = np.asarray(off, np.int64)
        return L.akmc_select_scratch_bytes(A._ptr(a), len(a) - 1)

    one = nbytes([0, 8192])
    assert one > 0
    assert nbytes([0, 8192 * 200 + 1]) > one                # 201 parts
    assert nbytes([0, 0, 5, 5]) > 0                        # empty segments are allowed
    assert nbytes([0, 5, 3]) == 0                          # decreasing
    assert nbytes([0, (1 << 30) + 1]) == 0                 # longer than 2^30 logits


def test_noalloc_wrapper_rejects_host_tensors_before_any_call():
    # the argument checks run on the host before the library is called: host
    # tensors, a short lattice buffer and a non-tensor are refused without a GPU
    torch = pytest.importorskip("torch")
    out = torch.zeros(8, dtype=torch.int64)
    with pytest.raises(ValueError, match="CUDA uint8"):
        A.cluster_hist_noalloc(torch.zeros(2 * 4 ** 3, dtype=torch.uint8), 4, 0, out)
    with pytest.raises(TypeError):
        A.cluster_hist_noalloc(np.zeros(2 * 4 ** 3, np.uint8), 4, 0, out)
