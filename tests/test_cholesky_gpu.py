"""dd Rpotrf / Rpotrs and the continuous-batching SPD-solve server (GPU).

Pins: exact recovery of an integer Cholesky factor (bit-exact), LAPACK test
ratios (< 30, the manual's LAPACK test threshold) on an SPD matrix of
condition ~1e20 with the residuals evaluated by the oracle's exact tier,
agreement with the oracle's solution within cond * eps, LAPACK info for
non-positive-definite input; the server's results are bitwise the same for a
request served alone and in a mix, and agree with the single-matrix routines.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import datagen
import oracle
from ddcheck import EPS_DD
from gpucase import dev, host

pytestmark = pytest.mark.gpu


def gpu_potrf(mp, uplo, Fh, Fl):
    n = Fh.shape[0]
    F = dev((Fh, Fl))
    info = torch.zeros(1, dtype=torch.int64, device="cuda")
    mp.mp_dd_Rpotrf(uplo, n, F, n, info)
    torch.cuda.synchronize()
    return F, int(info.item())


@pytest.mark.parametrize("uplo", ["U", "L"])
@pytest.mark.parametrize("n", [5, 64, 130])
def test_integer_factor_recovered_exactly(cuda_lib, uplo, n):
    g = datagen.rng(600 + n)
    U = np.triu(g.integers(-3, 4, (n, n))).astype(np.float64)
    np.fill_diagonal(U, g.integers(1, 5, n))
    Fm = U.T @ U
    assert np.abs(Fm).max() < 2 ** 52
    F, info = gpu_potrf(cuda_lib, uplo, np.asfortranarray(Fm), np.zeros((n, n), order="F"))
    assert info == 0
    fh, fl = host(F)
    if uplo == "U":
        assert np.array_equal(np.triu(fh), U) and not np.triu(fl).any()
    else:
        assert np.array_equal(np.tril(fh), U.T) and not np.tril(fl).any()


def test_not_positive_definite_info(cuda_lib):
    Fm = np.diag([4.0, 9.0, -1.0, 16.0])
    _, info = gpu_potrf(cuda_lib, "U", np.asfortranarray(Fm), np.zeros((4, 4), order="F"))
    assert info == 3
    n = 150
    Fm = np.eye(n) * 4.0
    Fm[99, 99] = -5.0                  # the leading minor of order 100 fails (block 2)
    _, info = gpu_potrf(cuda_lib, "L", np.asfortranarray(Fm), np.zeros((n, n), order="F"))
    assert info == 100


def spd_problem(seed, n):
    G, B = datagen.spd_request(seed, n)
    Fd = oracle.dd_syrk("U", "N", (1.0, 0.0), G, (0.0, 0.0),
                        (np.zeros((n, n), order="F"), np.zeros((n, n), order="F")))
    Fs = tuple(np.asfortranarray(np.triu(P) + np.triu(P, 1).T) for P in Fd)
    return G, B, Fs


@pytest.mark.parametrize("uplo", ["U", "L"])
def test_ill_conditioned_lapack_ratios_and_oracle(cuda_lib, uplo):
    n = 150
    G, B, Fs = spd_problem(610, n)
    F, info = gpu_potrf(cuda_lib, uplo, *Fs)
    assert info == 0
    fh, fl = host(F)
    Ut = (np.triu(fh), np.triu(fl)) if uplo == "U" else (np.tril(fh).T.copy(order="F"),
                                                         np.tril(fl).T.copy(order="F"))
    rr, cc = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    R = oracle.exact_gemm_entries("T", "N", n, (1.0, 0.0), Ut, Ut, (-1.0, 0.0), Fs,
                                  rr.ravel(), cc.ravel())
    fn = np.abs(Fs[0]).sum(axis=0).max()
    ratio_f = np.abs(R[0].reshape(n, n)).sum(axis=0).max() / (n * fn * EPS_DD)
    assert ratio_f < 30
    X = dev(B)
    cuda_lib.mp_dd_Rpotrs(uplo, n, 4, F, n, X, n)
    xh, xl = host(X)
    rr, cc = np.meshgrid(np.arange(n), np.arange(4), indexing="ij")
    R = oracle.exact_gemm_entries("N", "N", n, (-1.0, 0.0), Fs, (xh, xl), (1.0, 0.0), B,
                                  rr.ravel(), cc.ravel())
    xn = np.abs(xh).sum(axis=0).max()
    ratio_s = np.abs(R[0].reshape(n, 4)).sum(axis=0).max() / (fn * xn * EPS_DD)
    assert ratio_s < 30
    # the oracle's own factor-and-solve agrees to cond(F) * eps
    oh, ol, oinfo = oracle.dd_potrf("U", Fs)
    assert oinfo == 0
    Xo = oracle.dd_potrs("U", (oh, ol), B)
    rel = np.abs((xh - Xo[0]) + (xl - Xo[1])).max() / np.abs(Xo[0]).max()
    assert rel < 1e20 * EPS_DD * 100


def make_requests(seed, sizes):
    from paper_2109_13406_gb300.server import Request

    reqs = []
    for i, n in enumerate(sizes):
        G, B = datagen.spd_request(seed + i, int(n))
        reqs.append(Request(rid=i, n=int(n), G=G, B=B, arrival=0.002 * i))
    return reqs


def test_server_alone_equals_mix_bitwise(cuda_lib):
    from paper_2109_13406_gb300.server import SpdServer

    # n >= 256 takes the tensor-core (sliced) Rsyrk, smaller n the FP64 one
    sizes = [64, 100, 300, 70, 200, 90, 64, 260]
    mix = SpdServer(slots=5).serve(make_requests(620, sizes))
    assert sorted(r.rid for r in mix) == list(range(len(sizes)))
    by_id = {r.rid: r for r in mix}
    for i in (0, 2, 4, 7):
        alone = SpdServer().serve([make_requests(620, sizes)[i]])[0]
        assert alone.info == 0 and by_id[i].info == 0
        assert np.array_equal(alone.X[0], by_id[i].X[0])
        assert np.array_equal(alone.X[1], by_id[i].X[1])


def test_server_tensor_core_trailing_updates(cuda_lib):
    """Trailing updates through the residue-form Rgemm (forced on for every
    trailing block of 64 rows or more): bitwise the same alone and in a mix,
    the LAPACK ratio < 30, and the same solution as the FP64 updates within
    what the condition of F (~1e20) allows."""
    from paper_2109_13406_gb300.server import SpdServer, residual_ratio

    sizes = [300, 64, 260, 200]
    mix = SpdServer(slots=3, crt_min_rest=64).serve(make_requests(650, sizes))
    by_id = {r.rid: r for r in mix}
    assert all(r.info == 0 for r in mix)
    for i in (0, 2):
        alone = SpdServer(crt_min_rest=64).serve([make_requests(650, sizes)[i]])[0]
        assert np.array_equal(alone.X[0], by_id[i].X[0])
        assert np.array_equal(alone.X[1], by_id[i].X[1])
        fp64 = SpdServer(crt_min_rest=10 ** 9).serve([make_requests(650, sizes)[i]])[0]
        rel = np.abs((fp64.X[0] - alone.X[0]) + (fp64.X[1] - alone.X[1])).max()
        assert rel <= 1e20 * EPS_DD * 100 * np.abs(fp64.X[0]).max()
    n = sizes[0]
    G, B = datagen.spd_request(650, n)
    F = cuda_lib.dd_empty(n, n, fill=0.0)
    cuda_lib.mp_dd_Rsyrk("U", "N", n, 2 * n, (1.0, 0.0), dev(G), n, (0.0, 0.0), F, n)
    fh, fl = host(F)
    Fs = (np.triu(fh) + np.triu(fh, 1).T, np.triu(fl) + np.triu(fl, 1).T)
    assert residual_ratio(Fs, by_id[0].X, B, cuda_lib) < 30


@pytest.mark.parametrize("crt_min_rest", [64, 10 ** 9])
def test_server_group_sizes_agree(cuda_lib, crt_min_rest):
    """Groups of 4 blocks (row-block updates of depth up to 192, trailing
    updates of depth 256) and groups of 1 (rank-64 right-looking updates),
    with the updates in residue form or in FP64: the same solution within
    what cond(F) ~1e20 allows, and the LAPACK ratio < 30."""
    from paper_2109_13406_gb300.server import SpdServer, residual_ratio

    n = 520
    reqs = lambda: make_requests(660, [n])
    g4 = SpdServer(crt_min_rest=crt_min_rest, group=4).serve(reqs())[0]
    g1 = SpdServer(crt_min_rest=crt_min_rest, group=1).serve(reqs())[0]
    assert g4.info == 0 and g1.info == 0
    rel = np.abs((g1.X[0] - g4.X[0]) + (g1.X[1] - g4.X[1])).max()
    assert rel <= 1e20 * EPS_DD * 100 * np.abs(g1.X[0]).max()
    G, B = datagen.spd_request(660, n)
    F = cuda_lib.dd_empty(n, n, fill=0.0)
    cuda_lib.mp_dd_Rsyrk("U", "N", n, 2 * n, (1.0, 0.0), dev(G), n, (0.0, 0.0), F, n)
    fh, fl = host(F)
    Fs = (np.triu(fh) + np.triu(fh, 1).T, np.triu(fl) + np.triu(fl, 1).T)
    assert residual_ratio(Fs, g4.X, B, cuda_lib) < 30


@pytest.mark.parametrize("n", [130, 300])
def test_server_matches_single_matrix_routines(cuda_lib, n):
    from paper_2109_13406_gb300.server import SpdServer

    r = SpdServer().serve(make_requests(630, [n]))[0]
    G, B = datagen.spd_request(630, n)
    Gd = dev(G)
    F = cuda_lib.dd_empty(n, n, fill=0.0)
    cuda_lib.mp_dd_Rsyrk("U", "N", n, 2 * n, (1.0, 0.0), Gd, n, (0.0, 0.0), F, n)
    info = torch.zeros(1, dtype=torch.int64, device="cuda")
    cuda_lib.mp_dd_Rpotrf("U", n, F, n, info)
    X = dev(B)
    cuda_lib.mp_dd_Rpotrs("U", n, 4, F, n, X, n, info)
    xh, xl = host(X)
    rel = np.abs((xh - r.X[0]) + (xl - r.X[1])).max() / np.abs(xh).max()
    assert rel < 1e20 * EPS_DD * 100


def test_server_admission_respects_budget_and_slots(cuda_lib):
    from paper_2109_13406_gb300.server import SpdServer

    reqs = make_requests(640, [64, 80, 96, 64, 72, 88])
    budget = 2.5 * max(r.footprint() for r in reqs)
    srv = SpdServer(budget_bytes=budget, slots=2)
    done = srv.serve(reqs)
    assert len(done) == 6 and srv.max_active <= 2 and srv.used == 0
    assert all(r.info == 0 for r in done)


@pytest.mark.parametrize("nb", [64, 37])
def test_diag_batch_independent_of_cluster_size(cuda_lib, nb):
    """One diagonal block runs on a cluster of 8, 4, 2 or 1 CTAs depending on
    how many blocks a launch holds; each block's factor is the same bits in
    every configuration and equals Rpotrf's."""
    from paper_2109_13406_gb300 import _abi

    mp = cuda_lib
    _, _, Fs = spd_problem(612, nb)
    ref, info = gpu_potrf(mp, "L", *Fs)
    assert info == 0
    ref = host(ref)
    for count in (1, 30, 60, 160):              # clusters of 8, 4, 2, 1
        mats = [dev(Fs) for _ in range(count)]
        infos = torch.zeros(count, dtype=torch.int64, device="cuda")
        blob = b""
        for i, M in enumerate(mats):
            d = _abi.MpDDPotrfDiagDesc()
            d.a_hi, d.a_lo = M[0].data_ptr(), M[1].data_ptr()
            d.lda, d.n, d.offset, d.lower = nb, nb, 0, 1
            d.info = infos.data_ptr() + 8 * i
            blob += bytes(d)
        descs = torch.frombuffer(bytearray(blob), dtype=torch.uint8).cuda()
        mp.mp_dd_potrf_diag_batch(count, descs)
        torch.cuda.synchronize()
        assert not infos.any()
        for M in (mats[0], mats[-1]):
            h, l = host(M)
            assert np.array_equal(np.tril(h), np.tril(ref[0])), count
            assert np.array_equal(np.tril(l), np.tril(ref[1])), count


def _oracle_residual_ratio(Fs, X, B):
    """LAPACK ratio ||B - F X||_1 / (||F||_1 ||X||_1 eps_dd) with the residual
    from the oracle's exact tier (F symmetric, both triangles given)."""
    n, nrhs = X[0].shape
    rr, cc = np.meshgrid(np.arange(n), np.arange(nrhs), indexing="ij")
    R = oracle.exact_gemm_entries("N", "N", n, (-1.0, 0.0), Fs, X, (1.0, 0.0), B, rr.ravel(),
                                  cc.ravel())
    fn = np.abs(Fs[0]).sum(axis=0).max()
    xn = np.abs(X[0]).sum(axis=0).max()
    return np.abs(R[0].reshape(n, nrhs)).sum(axis=0).max() / (fn * xn * EPS_DD)


@pytest.mark.parametrize("crt_min_rest", [512, 64])
def test_served_solutions_against_the_oracle(cuda_lib, crt_min_rest):
    """Requests served in one mix -- F = G G^T on the tensor cores for
    n >= 256, trailing updates in residue form for 512+ (or, forced, 64+)
    columns and on the FP64 pipe below -- checked against the oracle: the
    residual of each served solution by the exact tier (LAPACK ratio < 30,
    the manual's LAPACK test threshold) with the oracle's own F, and the
    oracle's own factor-and-solve within cond(F) eps (cond ~1e20)."""
    from paper_2109_13406_gb300.server import SpdServer

    sizes = [96, 300, 640]
    done = SpdServer(slots=3, crt_min_rest=crt_min_rest).serve(make_requests(670, sizes))
    by_id = {r.rid: r for r in done}
    for i, n in enumerate(sizes):
        r = by_id[i]
        assert r.info == 0
        G, B, Fs = spd_problem(670 + i, n)
        assert _oracle_residual_ratio(Fs, r.X, B) < 30
        oh, ol, oinfo = oracle.dd_potrf("U", Fs)
        assert oinfo == 0
        Xo = oracle.dd_potrs("U", (oh, ol), B)
        rel = np.abs((r.X[0] - Xo[0]) + (r.X[1] - Xo[1])).max() / np.abs(Xo[0]).max()
        assert rel < 1e20 * EPS_DD * 100
