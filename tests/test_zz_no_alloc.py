"""The allocation-free query entry point (nbvh_query_rays_static).

Some callers cannot allocate device memory themselves, for example a renderer
or plug-in whose GPU memory belongs to a host application's fixed-budget
arena. For them the library keeps the query's scratch in a built-in device
array. This test calls that entry point through the C ABI twice in a row and
checks each result against the ordinary entry point, which uses a
caller-provided workspace, and checks that an oversized request is refused.
This file is collected last, and it builds everything it needs itself, so it
also passes when run alone in a fresh process."""
import numpy as np
import pytest

from gpu_cases import Built, make_case
from paper_2405_16237_b300 import nbvh as B

pytestmark = pytest.mark.gpu


def _compare(got, ref):
    # the same kernels on the same inputs (a row's result does not depend on
    # where it is evaluated), so any difference would be state left in the
    # shared scratch: bit-for-bit equality
    import torch
    for k in ref:
        assert torch.equal(got[k], ref[k]), k


@pytest.mark.parametrize("mlp_prec", [B.FP32, B.FP16])
def test_static_scratch_query_matches_workspace_query(mlp_prec):
    import torch
    assert torch.cuda.is_available()
    b = Built(make_case("random_tris_c0", table_scale=1.0, mlp_gain=2.0))
    desc = b.with_prec(mlp_prec)
    max_segs = 20
    ref = B.query_rays(desc, b.table, b.mlp, b.nodes, b.leaves["n_nodes"], b.rays, max_segs)
    assert B.device_status() == 0
    assert ref["hit"].cpu().numpy().sum() > 0
    outs = [B.new_hits(b.rays["ox"].numel()) for _ in range(2)]  # allocated before the calls
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for out in outs:
        B.query_rays_static(desc, b.table, b.mlp, b.nodes, b.leaves["n_nodes"], b.rays, max_segs, out=out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0  # the calls allocated no device memory
    assert B.device_status() == 0
    for out in outs:
        _compare(out, ref)


def test_static_scratch_rejects_oversized_requests():
    import torch
    b = Built(make_case("random_tris_c0"))
    n = b.rays["ox"].numel()
    # 4096 rays need ~ n * 12 * max_segs bytes of segment lists: pick max_segs past the capacity
    max_segs = 4000
    assert B.query_workspace_size(b.desc, n, max_segs) > B.STATIC_SCRATCH_BYTES
    with pytest.raises(B.NBVHError) as e:
        B.query_rays_static(b.desc, b.table, b.mlp, b.nodes, b.leaves["n_nodes"], b.rays, max_segs)
    assert e.value.code == 4
    torch.cuda.synchronize()
