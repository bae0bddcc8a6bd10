"""GPU parity of the site tables and of Q = gamma5 D_W (Sec. 2.1) against the oracle,
through the C-ABI: bit-exact tables, FP64 Q <= 1e-12, FP32 Q <= 1e-5 (relative L2),
FP16-storage Q with its measured error stated, for every link form."""
import numpy as np
import pytest

import synth
from oracle import geometry, wilson
from tests.gpu_util import dev, host, rel

pytestmark = pytest.mark.gpu
M = -1.4
TOL = {0: 1e-12, 1: 1e-5, 2: 2e-3}


@pytest.fixture(scope="module")
def nd():
    import paper_1010_5636_gb300 as nd
    nd.lib()
    return nd


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 4, 4, 4), (4, 6, 2, 8), (6, 4, 4, 6), (16, 16, 16, 32)])
def test_eo_tables_bit_exact(nd, dims):
    import torch
    ctx = nd.nd_create(dims)
    try:
        V = int(np.prod(dims))
        l2e = torch.empty(V, dtype=torch.int32, device="cuda")
        nbr = torch.empty((8, V), dtype=torch.int32, device="cuda")
        nd.nd_eo_tables(ctx, l2e, nbr)
        torch.cuda.synchronize()
        assert np.array_equal(host(l2e), geometry.lex_to_eo(dims))
        assert np.array_equal(host(nbr), geometry.neighbour_eo(dims))
    finally:
        nd.nd_destroy(ctx)


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_pack_round_trip(nd, prec):
    dims = (4, 6, 2, 8)
    psi = synth.spinor(dims, seed=1)
    ctx = nd.nd_create(dims)
    try:
        f = dev(psi)
        import torch
        buf = torch.empty(nd.nd_spinor_bytes(ctx, prec), dtype=torch.uint8, device="cuda")
        nd.nd_pack_spinor(ctx, buf, f, prec)
        back = torch.empty_like(f)
        nd.nd_unpack_spinor(ctx, back, buf, prec)
        torch.cuda.synchronize()
        if prec == 0:
            assert np.array_equal(host(back), psi)
        else:
            assert rel(host(back), psi) < (1e-7 if prec == 1 else 1e-3)
    finally:
        nd.nd_destroy(ctx)


def _q_case(nd, dims, kind, prec, recon, antiperiodic=False, seed=0):
    import torch
    U = synth.gauge_field(dims, kind, seed=seed, eps=0.3)
    psi = synth.spinor(dims, seed=1)
    expect = wilson.apply_Q(U, psi, dims, M, antiperiodic)
    ctx = nd.nd_create(dims, antiperiodic_t=antiperiodic, m=M)
    try:
        rc = [0, 0, 0]
        rc[prec] = recon
        nd.nd_set_links(ctx, dev(U), rc)
        inb = torch.empty(nd.nd_spinor_bytes(ctx, prec), dtype=torch.uint8, device="cuda")
        outb = torch.empty_like(inb)
        nd.nd_pack_spinor(ctx, inb, dev(psi), prec)
        nd.nd_apply_Q(ctx, outb, inb, prec)
        got = torch.empty((int(np.prod(dims)), 4, 3), dtype=torch.complex128, device="cuda")
        nd.nd_unpack_spinor(ctx, got, outb, prec)
        torch.cuda.synchronize()
        return rel(host(got), expect)
    finally:
        nd.nd_destroy(ctx)


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("recon", [18, 12, 8])
@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 4, 6), (4, 6, 2, 8)])
def test_Q_haar(nd, prec, recon, dims):
    err = _q_case(nd, dims, "haar", prec, recon)
    assert err <= TOL[prec], err


@pytest.mark.parametrize("prec,recon", [(0, 18), (1, 12), (1, 8), (2, 12)])
def test_Q_antiperiodic(nd, prec, recon):
    assert _q_case(nd, (4, 4, 2, 6), "haar", prec, recon, antiperiodic=True) <= TOL[prec]


@pytest.mark.parametrize("prec", [0, 1])
def test_Q_free_field_recon12(nd, prec):
    assert _q_case(nd, (4, 4, 4, 4), "unit", prec, 12) <= TOL[prec]


def test_recon8_rejects_unit_links(nd):
    dims = (2, 2, 2, 2)
    ctx = nd.nd_create(dims)
    try:
        with pytest.raises(nd.NdError) as e:
            nd.nd_set_links(ctx, dev(synth.gauge_field(dims, "unit")), (0, 8, 0))
        assert e.value.status == nd.ND_ERR_INVALID_ARG
    finally:
        nd.nd_destroy(ctx)


@pytest.mark.parametrize("parity", [0, 1])
@pytest.mark.parametrize("diag", [2.6, 0.0])
def test_Q_parity_block(nd, parity, diag):
    import torch
    dims = (4, 4, 6, 4)
    V = int(np.prod(dims))
    U = synth.gauge_field(dims, "near_identity", seed=0, eps=0.3)
    psi = synth.spinor(dims, seed=2)
    full = wilson.apply_Q(U, psi, dims, M)
    g5psi = psi.copy()
    g5psi[:, 2:] *= -1
    expect = full - (4 + M - diag) * g5psi
    par = geometry.coords(dims).sum(axis=1) % 2
    ctx = nd.nd_create(dims, m=M)
    try:
        nd.nd_set_links(ctx, dev(U), (18, 12, 0))
        for prec in (0, 1):
            inb = torch.empty(nd.nd_spinor_bytes(ctx, prec), dtype=torch.uint8, device="cuda")
            outb = torch.zeros_like(inb)
            nd.nd_pack_spinor(ctx, inb, dev(psi), prec)
            nd.nd_apply_Q_parity(ctx, outb, inb, prec, parity, diag)
            got = torch.empty((V, 4, 3), dtype=torch.complex128, device="cuda")
            nd.nd_unpack_spinor(ctx, got, outb, prec)
            torch.cuda.synchronize()
            g = host(got)[par == parity]
            assert rel(g, expect[par == parity]) <= TOL[prec]
    finally:
        nd.nd_destroy(ctx)


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_pack_round_trip_f32_canonical(nd, prec):
    """Canonical complex64 fields: FP64 and FP32 internal storage carry them bit-exactly, FP16
    to its storage precision; the FP32 form of a packed FP64 field is its rounding."""
    import torch
    dims = (4, 6, 2, 8)
    psi = synth.spinor(dims, seed=1)
    psi32 = psi.astype(np.complex64)
    ctx = nd.nd_create(dims)
    try:
        f = torch.from_numpy(psi32).cuda()
        buf = torch.empty(nd.nd_spinor_bytes(ctx, prec), dtype=torch.uint8, device="cuda")
        nd.nd_pack_spinor_f32(ctx, buf, f, prec)
        back = torch.empty_like(f)
        nd.nd_unpack_spinor_f32(ctx, back, buf, prec)
        torch.cuda.synchronize()
        if prec in (0, 1):
            assert np.array_equal(host(back), psi32)
        else:
            assert rel(host(back), psi32) < 1e-3
        if prec == 0:
            nd.nd_pack_spinor(ctx, buf, dev(psi), 0)
            nd.nd_unpack_spinor_f32(ctx, back, buf, 0)
            torch.cuda.synchronize()
            assert np.array_equal(host(back), psi32)
    finally:
        nd.nd_destroy(ctx)


@pytest.mark.parametrize("dims", [(32, 16, 16, 16), (48, 24, 24, 24), (64, 32, 32, 32)])
def test_Q_full_size_fp32(nd, dims):
    """The bench's lattices (near-identity links, as in the bandwidth sweep), whole-field parity."""
    assert _q_case(nd, dims, "near_identity", 1, 12) <= TOL[1]
    assert _q_case(nd, dims, "near_identity", 1, 8) <= TOL[1]


@pytest.mark.parametrize("recon", [18, 12, 8])
def test_Q_full_size_fp16(nd, recon):
    """FP16 storage with a per-site FP32 scale on the 24^3 x 48 sweep lattice.  No parity threshold
    is set for this form; its error against the oracle is printed and held to 2e-3."""
    err = _q_case(nd, (48, 24, 24, 24), "near_identity", 2, recon)
    print(f"FP16-{recon} Q on 24^3 x 48: relative L2 error {err:.2e} vs the oracle")
    assert err <= TOL[2], err


def test_Q_full_size_fp64(nd):
    assert _q_case(nd, (64, 32, 32, 32), "near_identity", 0, 18) <= TOL[0]


def test_Q_canonical(nd):
    import torch
    dims = (4, 4, 4, 6)
    U = synth.gauge_field(dims, "haar", seed=4)
    psi = synth.spinor(dims, seed=5)
    ctx = nd.nd_create(dims, m=M)
    try:
        nd.nd_set_links(ctx, dev(U), (18, 0, 0))
        out = torch.empty_like(dev(psi))
        nd.nd_apply_Q_canonical(ctx, out, dev(psi))
        torch.cuda.synchronize()
        assert rel(host(out), wilson.apply_Q(U, psi, dims, M)) <= 1e-12
    finally:
        nd.nd_destroy(ctx)


@pytest.mark.parametrize("prec,recon", [(0, 18), (1, 12), (1, 18), (2, 12)])
@pytest.mark.parametrize("nrhs", [2, 5, 12])
def test_Q_multi_rhs(nd, prec, recon, nrhs):
    """nrhs fields in one launch (links shared) equal nrhs single applications and the oracle."""
    import torch
    dims = (6, 4, 4, 6)
    V = int(np.prod(dims))
    U = synth.gauge_field(dims, "haar", seed=0)
    psi = synth.spinor(dims, seed=3, nrhs=nrhs)
    ctx = nd.nd_create(dims, m=M)
    try:
        rc = [0, 0, 0]
        rc[prec] = recon
        nd.nd_set_links(ctx, dev(U), rc)
        sb = nd.nd_spinor_bytes(ctx, prec)
        inb = torch.empty(sb * nrhs, dtype=torch.uint8, device="cuda")
        nd.nd_pack_spinor(ctx, inb, dev(psi), prec, nrhs)
        outb = torch.empty_like(inb)
        nd.nd_apply_Q(ctx, outb, inb, prec, nrhs)
        one = torch.empty_like(inb)
        for r in range(nrhs):
            nd.nd_apply_Q(ctx, one[r * sb:(r + 1) * sb], inb[r * sb:(r + 1) * sb], prec, 1)
        got = torch.empty((nrhs, V, 4, 3), dtype=torch.complex128, device="cuda")
        ref = torch.empty_like(got)
        nd.nd_unpack_spinor(ctx, got, outb, prec, nrhs)
        nd.nd_unpack_spinor(ctx, ref, one, prec, nrhs)
        torch.cuda.synchronize()
        # the autotuner may give the single launches another work split (another summation
        # order): two valid results agree to the precision's rounding, FP16 storage to ~1e-3
        assert rel(host(got), host(ref)) <= {0: 1e-15, 1: 1e-6, 2: 2e-3}[prec]
        exp = wilson.apply_Q(U, psi, dims, M)
        assert rel(host(got), exp) <= TOL[prec]
    finally:
        nd.nd_destroy(ctx)


def test_Q_multi_rhs_overlap_rejected(nd):
    import torch
    dims = (4, 4, 4, 4)
    ctx = nd.nd_create(dims, m=M)
    try:
        nd.nd_set_links(ctx, dev(synth.gauge_field(dims, "haar", seed=0)), (0, 12, 0))
        sb = nd.nd_spinor_bytes(ctx, 1)
        buf = torch.zeros(sb * 3, dtype=torch.uint8, device="cuda")
        with pytest.raises(nd.NdError) as e:
            nd.nd_apply_Q(ctx, buf[sb:], buf[:2 * sb], 1, 2)
        assert e.value.status == nd.ND_ERR_INVALID_ARG
    finally:
        nd.nd_destroy(ctx)


@pytest.mark.parametrize("prec,recon", [(1, 12), (0, 18), (2, 18)])
def test_Q_batched_lattices(nd, prec, recon):
    """One persistent launch over lattices of different sizes and RHS counts equals per-lattice Q."""
    import torch
    shapes = [((4, 4, 4, 4), 2), ((6, 4, 4, 6), 3), ((4, 6, 2, 8), 5)]
    ctxs, ins, outs, refs, canon = [], [], [], [], []
    try:
        for k, (dims, nr) in enumerate(shapes):
            U = synth.gauge_field(dims, "haar", seed=10 + k)
            ctx = nd.nd_create(dims, m=M)
            rc = [0, 0, 0]
            rc[prec] = recon
            nd.nd_set_links(ctx, dev(U), rc)
            psi = synth.spinor(dims, seed=20 + k, nrhs=nr)
            sb = nd.nd_spinor_bytes(ctx, prec)
            a = torch.empty(sb * nr, dtype=torch.uint8, device="cuda")
            nd.nd_pack_spinor(ctx, a, dev(psi), prec, nr)
            ref = torch.empty_like(a)
            nd.nd_apply_Q(ctx, ref, a, prec, nr)
            ctxs.append(ctx)
            ins.append(a)
            outs.append(torch.empty_like(a))
            refs.append(ref)
            canon.append((U, psi, dims, nr))
        nd.nd_apply_Q_batched(ctxs, outs, ins, [s[1] for s in shapes], prec)
        for ctx, o, r, (U, psi, dims, nr) in zip(ctxs, outs, refs, canon):
            V = int(np.prod(dims))
            got = torch.empty((nr, V, 4, 3), dtype=torch.complex128, device="cuda")
            exp = torch.empty_like(got)
            nd.nd_unpack_spinor(ctx, got, o, prec, nr)
            nd.nd_unpack_spinor(ctx, exp, r, prec, nr)
            torch.cuda.synchronize()
            assert rel(host(got), host(exp)) <= {0: 1e-15, 1: 1e-6, 2: 2e-3}[prec]
            assert rel(host(got), wilson.apply_Q(U, psi, dims, M)) <= TOL[prec]
    finally:
        for c in ctxs:
            nd.nd_destroy(c)


def test_autotune_cache_file(nd, tmp_path):
    """The autotuner writes its choices to ND_AUTOTUNE_CACHE in a fresh process and reuses them."""
    import os
    import subprocess
    import sys
    cache = tmp_path / "tune.txt"
    code = ("import sys; sys.path.insert(0, %r); import torch, synth, paper_1010_5636_gb300 as nd; "
            "from tests.gpu_util import dev; d=(8,8,8,8); c=nd.nd_create(d); "
            "nd.nd_set_links(c, dev(synth.gauge_field(d,'haar',seed=0)), (0,12,0)); "
            "a=torch.zeros(nd.nd_spinor_bytes(c,1), dtype=torch.uint8, device='cuda'); b=torch.empty_like(a); "
            "nd.nd_apply_Q(c,b,a,1); nd.nd_apply_Q_parity(c,b,a,1,0,0.0); torch.cuda.synchronize()") % os.getcwd()
    env = dict(os.environ, ND_AUTOTUNE_CACHE=str(cache))
    subprocess.run([sys.executable, "-c", code], check=True, env=env, cwd=os.getcwd())
    lines = cache.read_text().split("\n")
    assert len([ln for ln in lines if ln.startswith("q:")]) == 2
    subprocess.run([sys.executable, "-c", code], check=True, env=env, cwd=os.getcwd())
    assert len([ln for ln in cache.read_text().split("\n") if ln.startswith("q:")]) == 2  # reused, not retuned


@pytest.mark.parametrize("krhs", [2, 3])
def test_Q_multi_rhs_per_thread(krhs):
    """Several RHS per thread sharing each link (ND_Q_KRHS, read once per process, hence a child
    process): FP32 and FP16 results equal single applications to the storage precision's rounding
    (the two kernels may contract the epilogue into fused multiply-adds differently) and match the
    oracle."""
    import os
    import subprocess
    import sys
    code = r'''
import sys, numpy as np, torch
sys.path.insert(0, %r)
import synth, paper_1010_5636_gb300 as nd
from oracle import wilson
from tests.gpu_util import dev, host, rel
dims = (4, 6, 4, 8)
V = int(np.prod(dims))
U = synth.gauge_field(dims, "haar", seed=0)
for prec, recon, tol in ((1, 12, 1e-5), (1, 18, 1e-5), (2, 12, 2e-3)):
    for nrhs in (2, 5, 7):
        psi = synth.spinor(dims, seed=3, nrhs=nrhs)
        ctx = nd.nd_create(dims, m=-1.4)
        rc = [0, 0, 0]; rc[prec] = recon
        nd.nd_set_links(ctx, dev(U), rc)
        sb = nd.nd_spinor_bytes(ctx, prec)
        a = torch.empty(sb * nrhs, dtype=torch.uint8, device="cuda")
        nd.nd_pack_spinor(ctx, a, dev(psi), prec, nrhs)
        b = torch.empty_like(a); one = torch.empty_like(a)
        nd.nd_apply_Q(ctx, b, a, prec, nrhs)
        for r in range(nrhs):
            nd.nd_apply_Q(ctx, one[r * sb:(r + 1) * sb], a[r * sb:(r + 1) * sb], prec, 1)
        got = torch.empty((nrhs, V, 4, 3), dtype=torch.complex128, device="cuda")
        ref = torch.empty_like(got)
        nd.nd_unpack_spinor(ctx, got, b, prec, nrhs)
        nd.nd_unpack_spinor(ctx, ref, one, prec, nrhs)
        torch.cuda.synchronize()
        assert rel(host(got), host(ref)) <= (1e-6 if prec == 1 else 1e-3), (prec, recon, nrhs)
        assert rel(host(got), wilson.apply_Q(U, psi, dims, -1.4)) <= tol
        nd.nd_destroy(ctx)
print("ok")
''' % os.getcwd()
    env = dict(os.environ, ND_Q_KRHS=str(krhs), ND_AUTOTUNE="0")
    r = subprocess.run([sys.executable, "-c", code], env=env, cwd=os.getcwd(), capture_output=True, text=True)
    assert r.returncode == 0 and "ok" in r.stdout, r.stderr[-2000:]
