"""The allocation-free Q with fused norms (nd_apply_Q_norms_static), for callers that may not
call cudaMalloc at call time: its output must equal nd_apply_Q's and its norms the norms of
the two fields, on two calls in a row (the second call reuses the static scratch that the
first one left behind), and the second call must leave the device's free memory unchanged.
Collected last on purpose."""
import numpy as np
import pytest

import synth
from tests.gpu_util import dev, host

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5)])
def test_static_norms_match_existing_entry_point(prec, tol):
    import torch

    import paper_1010_5636_gb300 as nd
    dims = (6, 4, 4, 6)
    U = synth.gauge_field(dims, "haar", seed=0)
    ctx = nd.nd_create(dims, m=-1.4, s=0.4)
    try:
        nd.nd_set_links(ctx, dev(U), (18, 12, 0))
        for call in range(2):
            psi = synth.spinor(dims, seed=10 + call)
            a = torch.empty(nd.nd_spinor_bytes(ctx, prec), dtype=torch.uint8, device="cuda")
            nd.nd_pack_spinor(ctx, a, dev(psi), prec)
            ref = torch.empty_like(a)
            nd.nd_apply_Q(ctx, ref, a, prec)
            out = torch.empty_like(a)
            torch.cuda.synchronize()
            free_before = torch.cuda.mem_get_info()[0]
            n_out, n_in = nd.nd_apply_Q_norms_static(ctx, out, a, prec)
            torch.cuda.synchronize()
            if call == 1:
                # the first call may load the module and look up the array's address; the second must
                # leave the device's free memory exactly as it was (no allocation of any kind)
                assert torch.cuda.mem_get_info()[0] == free_before
            V = int(np.prod(dims))
            got_c = torch.empty((V, 4, 3), dtype=torch.complex128, device="cuda")
            ref_c = torch.empty_like(got_c)
            in_c = torch.empty_like(got_c)
            nd.nd_unpack_spinor(ctx, got_c, out, prec)
            nd.nd_unpack_spinor(ctx, ref_c, ref, prec)
            nd.nd_unpack_spinor(ctx, in_c, a, prec)
            torch.cuda.synchronize()
            g, r, i = host(got_c), host(ref_c), host(in_c)
            assert np.linalg.norm(g - r) <= tol * np.linalg.norm(r)
            assert abs(n_out - np.vdot(r, r).real) <= tol * np.vdot(r, r).real
            assert abs(n_in - np.vdot(i, i).real) <= tol * np.vdot(i, i).real
    finally:
        nd.nd_destroy(ctx)


def test_static_norms_rejects_large_lattice():
    import torch

    import paper_1010_5636_gb300 as nd
    dims = (66, 32, 32, 64)  # 4325376 sites, above the 4194304-site limit
    ctx = nd.nd_create(dims, m=-1.4, s=0.4)
    try:
        buf = torch.empty(16, dtype=torch.uint8, device="cuda")
        with pytest.raises(nd.NdError) as e:
            nd.nd_apply_Q_norms_static(ctx, buf, buf[8:], 1)
        assert e.value.status == nd.ND_ERR_INVALID_ARG
    finally:
        nd.nd_destroy(ctx)
