"""The allocation-free cluster histogram entry point (akmc_cluster_hist_noalloc)
against the workspace-based one (akmc_cluster_hist).

The no-alloc variant exists for callers that cannot let a library allocate
device memory (their GPU memory is owned by another allocator, or they sit
on a latency-critical path); its scratch is a fixed device array inside the
library.  This file is collected last so that a failure here, in a run that
stops at the first failure, comes after every other test; it also passes
when run alone in a fresh process."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2604_24091_gb300 import AkmcError, Batch  # noqa: E402
from paper_2604_24091_gb300.akmc import cluster_hist_noalloc  # noqa: E402


def test_noalloc_cluster_hist_matches_workspace_entry_point(model):
    descs = [synth.VoxelDesc(10, 2, (0.10, 0.02, 0.02), 563.0, synth.PAIR_MODEL, synth.PREC_FP64, seed=71, uid=1),
             synth.VoxelDesc(32, 1, (0.02, 0.007, 0.014), 563.0, synth.EAM_MODEL, synth.PREC_SPLIT, seed=72, uid=2),
             synth.VoxelDesc(64, 1, (0.01, 0.0, 0.0), 563.0, synth.PAIR_MODEL, synth.PREC_FP64, seed=73, uid=3)]
    b = Batch(descs, model)
    b.step(400)
    # The first call runs on a fresh non-blocking stream: in a fresh process it is
    # the call that does the one-time set-up, and nothing orders that stream after
    # the set-up's copy unless the entry point waits for it.
    side = torch.cuda.Stream()
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5)
    # three calls in a row, different lattices and modes, sharing the static scratch;
    # the output starts as garbage, so the entry point must clear it itself
    for i, (v, mode) in enumerate(((0, 0), (2, 1), (1, 0))):
        s = b.read_state(v)["species"]
        dev = torch.from_numpy(s).cuda()
        out = torch.randint(-2 ** 62, 2 ** 62, (8,), dtype=torch.int64, device="cuda", generator=gen)
        torch.cuda.synchronize()
        if i == 0:
            with torch.cuda.stream(side):
                cluster_hist_noalloc(dev, descs[v].L, mode, out, stream=side)
            side.synchronize()
        else:
            cluster_hist_noalloc(dev, descs[v].L, mode, out)
        got = out.cpu().numpy().tolist()
        assert got == b.cluster_hist(v, mode).tolist()
        o = oracle.Voxel(descs[v], model)
        o.load(s, b.read_state(v)["vac_pos"])
        assert got == o.cluster_hist(mode)[0].tolist()


def test_noalloc_rejects_lattices_above_the_static_size():
    dev = torch.zeros(2 * 65 ** 3, dtype=torch.uint8, device="cuda")
    out = torch.zeros(8, dtype=torch.int64, device="cuda")
    with pytest.raises(AkmcError, match="outside"):
        cluster_hist_noalloc(dev, 65, 0, out)


def test_noalloc_rejects_short_or_misplaced_buffers():
    out = torch.zeros(8, dtype=torch.int64, device="cuda")
    short = torch.zeros(2 * 10 ** 3 - 1, dtype=torch.uint8, device="cuda")
    with pytest.raises(ValueError, match="fewer than"):
        cluster_hist_noalloc(short, 10, 0, out)
    ok = torch.zeros(2 * 10 ** 3, dtype=torch.uint8, device="cuda")
    with pytest.raises(ValueError, match="contiguous"):
        cluster_hist_noalloc(ok, 10, 0, torch.zeros(16, dtype=torch.int64, device="cuda")[::2])
    with pytest.raises(ValueError):
        cluster_hist_noalloc(ok, 10, 0, torch.zeros(8, dtype=torch.int64))
