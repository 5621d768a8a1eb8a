"""GPU parity of single hot-path operations (C ABI, FP64 mode) against the CPU oracle:
projected-Hamiltonian matvec, projected-operator updates, SVD split with truncation."""
import numpy as np
import pytest

import workloads as wl
from oracle import dmrg as O
from oracle.accsvd import accurate_svd
from tests import _layout as LY

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

pd = pytest.importorskip("paper_1301_3494_gb300")


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _bond_case(kind, m, seed):
    """Random bond sectors of total size ~m around a chain / cylinder MPO."""
    rng = np.random.default_rng(seed)
    if kind == "chain":
        mpo = wl.heisenberg_chain(40)
        j = 20
    elif kind == "cyl":
        mpo = wl.heisenberg_square_cylinder(6, 4)
        j = 11
    else:
        mpo = wl.tfim_chain(30, 1.0, 0.7)
        j = 15
    qn = list(mpo.site.qn)
    bonds = wl.bond_sectors(mpo.L, qn, 0, m, sigma=None if kind == "tfim" else 3.0)
    return mpo, qn, bonds[j], bonds[j + 2], bonds[j + 1], j, rng


@pytest.mark.parametrize("kind,m", [("chain", 40), ("chain", 300), ("cyl", 150), ("tfim", 150)])
def test_heff_apply_fp64_matches_oracle(kind, m):
    mpo, qn, bl, br, _, j, rng = _bond_case(kind, m, 1)
    W1, W2 = mpo.W[j], mpo.W[j + 1]
    f0, f1, f2 = mpo.flux[j], mpo.flux[j + 1], mpo.flux[j + 2]
    Lenv = LY.random_env(bl, f0, rng)
    Renv = LY.random_env(br, f2, rng)
    psi = {k: rng.standard_normal((bl[k[0]], br[k[0] + qn[k[1]] + qn[k[2]]])) for k in LY.psi_keys(bl, br, qn)}
    ref = O.heff_apply(Lenv, W1, f0, W2, f2, Renv, psi, qn)
    bond = pd.Bond(qn, bl, br, W1, f0, f1, W2, f2)
    Ld, Rd = _dev(LY.pack_env(Lenv, bl, f0)), _dev(LY.pack_env(Renv, br, f2))
    x = _dev(LY.pack_psi(psi, bl, br, qn))
    y = torch.zeros_like(x)
    flops = pd.heff_apply(bond, pd.FP64, Ld.data_ptr(), Rd.data_ptr(), x.data_ptr(), y.data_ptr())
    torch.cuda.synchronize()
    got = LY.unpack_psi(y.cpu().numpy(), bl, br, qn)
    scale = max(np.abs(v).max() for v in ref.values())
    for k in ref:
        assert np.abs(got[k] - ref[k]).max() <= 1e-12 * scale, k
    assert flops > 0


@pytest.mark.parametrize("kind,m", [("chain", 60), ("cyl", 200), ("tfim", 100)])
def test_env_updates_fp64_match_oracle(kind, m):
    mpo, qn, bl, _, bm, j, rng = _bond_case(kind, m, 2)
    W = mpo.W[j]
    fL, fR = mpo.flux[j], mpo.flux[j + 1]
    A = {k: rng.standard_normal((bl[k[0]], bm[k[0] + qn[k[1]]])) for k in LY.site_keys(bl, bm, qn)}
    Lin = LY.random_env(bl, fL, rng)
    ref = O.env_left(Lin, A, W, fL, fR, qn)
    bond = pd.Bond(qn, bl, bm, W, fL, fR)
    Lo = torch.zeros(len(LY.env_keys(bm, fR)) and sum(bm[q] * bm[q - int(fR[w])] for q, w in LY.env_keys(bm, fR)),
                     dtype=torch.float64, device="cuda")
    Lin_d, A_d = _dev(LY.pack_env(Lin, bl, fL)), _dev(LY.pack_site(A, bl, bm, qn))   # keep references alive
    pd.env_left(bond, pd.FP64, Lin_d.data_ptr(), A_d.data_ptr(), Lo.data_ptr())
    torch.cuda.synchronize()
    got = LY.unpack_env(Lo.cpu().numpy(), bm, fR)
    scale = max(np.abs(v).max() for v in ref.values())
    for k in LY.env_keys(bm, fR):
        r = ref.get(k, np.zeros_like(got[k]))
        assert np.abs(got[k] - r).max() <= 1e-12 * scale, k
    # right update through the same site
    Rin = LY.random_env(bm, fR, rng)
    refR = O.env_right(Rin, A, W, fL, fR, qn)
    Ro = torch.zeros(sum(bl[q] * bl[q - int(fL[w])] for q, w in LY.env_keys(bl, fL)), dtype=torch.float64, device="cuda")
    Rin_d = _dev(LY.pack_env(Rin, bm, fR))
    pd.env_right(bond, pd.FP64, Rin_d.data_ptr(), A_d.data_ptr(), Ro.data_ptr())
    torch.cuda.synchronize()
    gotR = LY.unpack_env(Ro.cpu().numpy(), bl, fL)
    scale = max(np.abs(v).max() for v in refR.values())
    for k in LY.env_keys(bl, fL):
        r = refR.get(k, np.zeros_like(gotR[k]))
        assert np.abs(gotR[k] - r).max() <= 1e-12 * scale, k


@pytest.mark.parametrize("plain", [0, 4])
@pytest.mark.parametrize("kind,m,mmax", [("chain", 60, 1000), ("chain", 200, 120), ("cyl", 160, 90), ("tfim", 80, 50)])
def test_svd_split_matches_oracle(kind, m, mmax, plain):
    """FP64 split (Jacobi on R^T from a Householder QR, or with plain = 4 on the sector matrices)
    against the oracle: block table, discarded weight, singular values, factors."""
    mpo, qn, bl, br, _, j, rng = _bond_case(kind, m, 3)
    # a wavefunction with a decaying spectrum (like a ground state)
    psi = {}
    for k in LY.psi_keys(bl, br, qn):
        a, c = bl[k[0]], br[k[0] + qn[k[1]] + qn[k[2]]]
        psi[k] = rng.standard_normal((a, c)) * np.exp(-0.05 * np.add.outer(np.arange(a), np.arange(c)))
    A, lam, B, counts, err = O.split_two_site(psi, bl, br, qn, mmax)
    bond = pd.Bond(qn, bl, br, mpo.W[j], mpo.flux[j], mpo.flux[j + 1])
    x = _dev(LY.pack_psi(psi, bl, br, qn))
    n = x.numel()
    Ad = torch.zeros(n + 16, dtype=torch.float64, device="cuda")
    Bd = torch.zeros(n + 16, dtype=torch.float64, device="cuda")
    ld = torch.zeros(n + 16, dtype=torch.float64, device="cuda")
    mid, tr = pd.svd_split(bond, x.data_ptr(), mmax, plain, Ad.data_ptr(), ld.data_ptr(), Bd.data_ptr())
    torch.cuda.synchronize()
    assert mid == counts                                   # block table bit-exact
    assert abs(tr - err) <= 1e-12 + 1e-9 * err
    lam_ref = np.concatenate([lam[q] for q in sorted(lam)])
    lam_gpu = ld.cpu().numpy()[: lam_ref.size]
    assert np.abs(lam_gpu - lam_ref).max() <= 1e-12
    # factors: orthonormal, and A diag(lam) B reproduces the oracle's truncated Psi
    Ag = LY.unpack_site(Ad.cpu().numpy(), bl, mid, qn)
    Bg = LY.unpack_site(Bd.cpu().numpy(), mid, br, qn)
    lg, off = {}, 0
    for q in sorted(mid):
        lg[q] = lam_gpu[off: off + mid[q]]
        off += mid[q]
    rec_g = O.two_site({k: v * lg[k[0] + qn[k[1]]][None, :] for k, v in Ag.items()}, Bg, qn)
    rec_o = O.two_site({k: v * lam[k[0] + qn[k[1]]][None, :] for k, v in A.items()}, B, qn)
    for k in rec_o:
        assert np.abs(rec_g[k] - rec_o[k]).max() <= 1e-11, k


@pytest.mark.parametrize("plain", [0, 4])
@pytest.mark.parametrize("kind,m,seed", [("chain", 60, 7), ("cyl", 120, 8)])
def test_svd_split_accurate_graded(kind, m, seed, plain):
    """Appendix accurate SVD (mode 1) on graded blocks D1 G D2 (rows graded over 7 decades,
    columns over 2): every singular value agrees with the oracle's accurate SVD to 1e-9 relative
    (the oracle's recursion is pinned against 60-digit arithmetic), the block table exactly, and
    the factors reproduce the oracle's Psi."""
    mpo, qn, bl, br, _, j, rng = _bond_case(kind, m, seed)
    psi = {}
    for k in LY.psi_keys(bl, br, qn):
        a, c = bl[k[0]], br[k[0] + qn[k[1]] + qn[k[2]]]
        d1 = 10.0 ** (-rng.uniform(0.0, 7.0, a))
        d2 = 10.0 ** (-rng.uniform(0.0, 2.0, c))
        psi[k] = d1[:, None] * rng.standard_normal((a, c)) * d2[None, :]
    A, lam, B, counts, err = O.split_two_site(psi, bl, br, qn, 10 ** 9, accurate_svd)
    bond = pd.Bond(qn, bl, br, mpo.W[j], mpo.flux[j], mpo.flux[j + 1])
    x = _dev(LY.pack_psi(psi, bl, br, qn))
    n = x.numel()
    Ad = torch.zeros(n + 16, dtype=torch.float64, device="cuda")
    Bd = torch.zeros(n + 16, dtype=torch.float64, device="cuda")
    ld = torch.zeros(n + 16, dtype=torch.float64, device="cuda")
    mid, tr = pd.svd_split(bond, x.data_ptr(), 10 ** 9, 1 + plain, Ad.data_ptr(), ld.data_ptr(), Bd.data_ptr())
    torch.cuda.synchronize()
    assert mid == counts
    lam_ref = np.concatenate([lam[q] for q in sorted(lam)])
    lam_gpu = ld.cpu().numpy()[: lam_ref.size]
    assert lam_ref.min() < 1e-6 * lam_ref.max()          # the recursion has work to do
    assert np.all(np.abs(lam_gpu - lam_ref) <= 1e-9 * lam_ref)
    Ag = LY.unpack_site(Ad.cpu().numpy(), bl, mid, qn)
    Bg = LY.unpack_site(Bd.cpu().numpy(), mid, br, qn)
    lg, off = {}, 0
    for q in sorted(mid):
        lg[q] = lam_gpu[off: off + mid[q]]
        off += mid[q]
    rec_g = O.two_site({k: v * lg[k[0] + qn[k[1]]][None, :] for k, v in Ag.items()}, Bg, qn)
    rec_o = O.two_site({k: v * lam[k[0] + qn[k[1]]][None, :] for k, v in A.items()}, B, qn)
    for k in rec_o:
        assert np.abs(rec_g[k] - rec_o[k]).max() <= 1e-12 * lam_ref.max(), k


@pytest.mark.parametrize("plain", [0, 4])
@pytest.mark.parametrize("kind,m,mmax", [("chain", 200, 120), ("cyl", 160, 90), ("cyl", 420, 300), ("tfim", 80, 50),
                                          ("chain", 3200, 2000)])
def test_svd_split_fp32_block_jacobi(kind, m, mmax, plain):
    """Mixed-precision split (FP32 block Jacobi, A re-orthonormalised in FP64) against the FP64
    oracle.  FP32 columns carry absolute errors ~eps_f32 * lambda_max and pairs stop rotating at a
    relative off-diagonal of 3e-5, so singular values agree to 1e-4 * lambda_max and the
    reconstruction to 2e-4 normwise; A is orthonormal to FP64
    accuracy; the block table equals the oracle's wherever the cut has a gap above that error."""
    mpo, qn, bl, br, _, j, rng = _bond_case(kind, m, 3)
    psi = {}
    for k in LY.psi_keys(bl, br, qn):
        a, c = bl[k[0]], br[k[0] + qn[k[1]] + qn[k[2]]]
        psi[k] = rng.standard_normal((a, c)) * np.exp(-0.02 * np.add.outer(np.arange(a), np.arange(c)))
    nrm = np.sqrt(sum((v ** 2).sum() for v in psi.values()))
    psi = {k: v / nrm for k, v in psi.items()}
    A, lam, B, counts, err = O.split_two_site(psi, bl, br, qn, mmax)
    lam_all = np.sort(np.concatenate(list(lam.values())))[::-1]
    bond = pd.Bond(qn, bl, br, mpo.W[j], mpo.flux[j], mpo.flux[j + 1])
    x = _dev(LY.pack_psi(psi, bl, br, qn))
    n = x.numel()
    Ad = torch.zeros(n + 16, dtype=torch.float64, device="cuda")
    Bd = torch.zeros(n + 16, dtype=torch.float64, device="cuda")
    ld = torch.zeros(n + 16, dtype=torch.float64, device="cuda")
    mid, tr = pd.svd_split(bond, x.data_ptr(), mmax, 2 + plain, Ad.data_ptr(), ld.data_ptr(), Bd.data_ptr())
    torch.cuda.synchronize()
    # the oracle's full spectrum decides whether the cut is resolvable in FP32
    full = O.split_two_site(psi, bl, br, qn, 10 ** 9)[1]
    spec = np.sort(np.concatenate(list(full.values())))[::-1]
    kept = int(sum(mid.values()))
    if len(spec) > mmax and spec[mmax - 1] - spec[mmax] > 1e-4 * spec[0] and spec[mmax - 1] > 1e-4 * spec[0]:
        assert mid == counts
    assert kept <= mmax
    lam_gpu = ld.cpu().numpy()[:kept]
    got = np.sort(lam_gpu)[::-1]
    assert np.abs(got - spec[:kept] / np.sqrt((spec[:kept] ** 2).sum())).max() <= 1e-4 * spec[0]
    Ag = LY.unpack_site(Ad.cpu().numpy(), bl, mid, qn)
    Bg = LY.unpack_site(Bd.cpu().numpy(), mid, br, qn)
    for q in mid:   # A^T A = 1 per middle sector, FP64 accuracy
        cols = [v for k, v in Ag.items() if k[0] + qn[k[1]] == q]
        M = np.concatenate(cols, axis=0)
        assert np.abs(M.T @ M - np.eye(M.shape[1])).max() <= 1e-12
    lg, off = {}, 0
    for q in sorted(mid):
        lg[q] = lam_gpu[off: off + mid[q]]
        off += mid[q]
    rec_g = O.two_site({k: v * lg[k[0] + qn[k[1]]][None, :] for k, v in Ag.items()}, Bg, qn)
    rec_o = O.two_site({k: v * lam[k[0] + qn[k[1]]][None, :] for k, v in A.items()}, B, qn)
    diff = sum(((rec_g.get(k, 0) - rec_o[k]) ** 2).sum() for k in rec_o)
    assert np.sqrt(diff) <= 2e-4 + 2 * np.sqrt(err)


@pytest.mark.parametrize("mode", [0, 2, 6])
def test_svd_split_batch_equals_single_splits(mode):
    """dmrg_svd_split_batch over four bonds of different shapes and charge sets (chain, cylinder,
    TFIM, a tiny chain bond; one grouped Jacobi launch over all their sectors) returns, bond by
    bond, what dmrg_svd_split returns for that bond alone -- same block table, discarded weight,
    lambda and factors -- and what the oracle returns: FP64 mode (0) to 1e-12; the FP32 block
    Jacobi (2, and 6 without the QR) to the FP32 split's bounds (lambda 1e-4 lambda_max, the
    reconstruction 2e-4 normwise), lambda to 5e-5 lambda_max of the single-bond FP32 run (the
    FP32 Jacobi stops at a relative off-diagonal of 3e-5, and the staging of a sector's columns,
    so the rounding of its rotations, follows the batch's largest sector)."""
    cases = [("chain", 200, 120), ("cyl", 420, 300), ("tfim", 80, 50), ("chain", 12, 6)]
    fp32 = (mode & 3) == 2
    bonds, xs, single, batch, refs, mmaxs = [], [], [], [], [], []
    for i, (kind, m, mmax) in enumerate(cases):
        mpo, qn, bl, br, _, j, rng = _bond_case(kind, m, 11 + i)
        psi = {}
        for k in LY.psi_keys(bl, br, qn):
            a, c = bl[k[0]], br[k[0] + qn[k[1]] + qn[k[2]]]
            psi[k] = rng.standard_normal((a, c)) * np.exp(-0.02 * np.add.outer(np.arange(a), np.arange(c)))
        nrm = np.sqrt(sum((v ** 2).sum() for v in psi.values()))
        psi = {k: v / nrm for k, v in psi.items()}
        bond = pd.Bond(qn, bl, br, mpo.W[j], mpo.flux[j], mpo.flux[j + 1])
        x = _dev(LY.pack_psi(psi, bl, br, qn))
        n = x.numel()
        s_bufs = [torch.zeros(n + 16, dtype=torch.float64, device="cuda") for _ in range(3)]
        b_bufs = [torch.zeros(n + 16, dtype=torch.float64, device="cuda") for _ in range(3)]
        mid, tr = pd.svd_split(bond, x.data_ptr(), mmax, mode, s_bufs[0].data_ptr(), s_bufs[1].data_ptr(),
                               s_bufs[2].data_ptr())
        single.append((mid, tr, s_bufs))
        batch.append(b_bufs)
        bonds.append(bond)
        xs.append(x)
        mmaxs.append(mmax)
        refs.append((qn, bl, br, O.split_two_site(psi, bl, br, qn, mmax),
                     O.split_two_site(psi, bl, br, qn, 10 ** 9)[1]))
    res = pd.svd_split_batch(bonds, [x.data_ptr() for x in xs], mmaxs, mode, [b[0].data_ptr() for b in batch],
                             [b[1].data_ptr() for b in batch], [b[2].data_ptr() for b in batch])
    torch.cuda.synchronize()
    assert len(res) == len(cases)
    for (mid_b, tr_b), (mid_s, tr_s, s_bufs), b_bufs, (qn, bl, br, ref, full), mmax in zip(
            res, single, batch, refs, mmaxs):
        A, lam, B, counts, err = ref
        spec = np.sort(np.concatenate(list(full.values())))[::-1]
        resolvable = len(spec) <= mmax or (spec[mmax - 1] - spec[mmax] > 1e-4 * spec[0]
                                           and spec[mmax - 1] > 1e-4 * spec[0])
        if not fp32 or resolvable:
            assert mid_b == counts
        assert mid_b == mid_s
        kept = int(sum(mid_b.values()))
        lam_b = b_bufs[1].cpu().numpy()[:kept]
        lam_s = s_bufs[1].cpu().numpy()[:kept]
        lam_ref = np.concatenate([lam[q] for q in sorted(lam)]) if not fp32 else None
        if fp32:
            assert np.abs(lam_b - lam_s).max() <= 5e-5 * spec[0]
            got = np.sort(lam_b)[::-1]
            assert np.abs(got - spec[:kept] / np.sqrt((spec[:kept] ** 2).sum())).max() <= 1e-4 * spec[0]
            assert abs(tr_b - tr_s) <= 1e-5
        else:
            assert np.abs(lam_b - lam_ref).max() <= 1e-12
            assert np.abs(lam_b - lam_s).max() <= 1e-13
            assert abs(tr_b - err) <= 1e-12 + 1e-9 * err
        Ab = LY.unpack_site(b_bufs[0].cpu().numpy(), bl, mid_b, qn)
        Bb = LY.unpack_site(b_bufs[2].cpu().numpy(), mid_b, br, qn)
        As = LY.unpack_site(s_bufs[0].cpu().numpy(), bl, mid_s, qn)
        Bs = LY.unpack_site(s_bufs[2].cpu().numpy(), mid_s, br, qn)
        lg, off = {}, 0
        for q in sorted(mid_b):
            lg[q] = lam_b[off: off + mid_b[q]]
            off += mid_b[q]
        ls, off = {}, 0
        for q in sorted(mid_s):
            ls[q] = lam_s[off: off + mid_s[q]]
            off += mid_s[q]
        rec_b = O.two_site({k: v * lg[k[0] + qn[k[1]]][None, :] for k, v in Ab.items()}, Bb, qn)
        rec_s = O.two_site({k: v * ls[k[0] + qn[k[1]]][None, :] for k, v in As.items()}, Bs, qn)
        rec_o = O.two_site({k: v * lam[k[0] + qn[k[1]]][None, :] for k, v in A.items()}, B, qn)
        if fp32:   # normwise
            d_bs = np.sqrt(sum(((rec_b.get(k, 0) - rec_s.get(k, 0)) ** 2).sum() for k in rec_o))
            d_bo = np.sqrt(sum(((rec_b.get(k, 0) - rec_o[k]) ** 2).sum() for k in rec_o))
            assert d_bs <= 2e-4 + 2 * np.sqrt(err)
            assert d_bo <= 2e-4 + 2 * np.sqrt(err)
        else:      # element by element
            for k in rec_o:
                assert np.abs(rec_b[k] - rec_s[k]).max() <= 1e-12, k
                assert np.abs(rec_b[k] - rec_o[k]).max() <= 1e-11, k


# ------------------------------------------------------------------------------------------
# Tensor-core (tcgen05) paths against the FP64 oracle, element by element and normwise.  Every
# product term L W1 W2 R x of an output element passes through at most four operand roundings
# (x, L and R to the operand type, the MPO-mixed intermediate Y to it as well) and FP32
# accumulation, so |y - y_ref| <= c u (|L| |W1| |W2| |R| |x|) elementwise, the right side being the
# oracle applied to absolute values; u = 2^-8 for bf16 (8 significant bits, round to nearest) and
# 2^-10 for tf32 (11 bits, the conversion may truncate), c = 8 (four roundings, twice over for
# margin; FP32 accumulation adds K 2^-24, below 1e-3 u).  Normwise: 2e-2 (bf16), 5e-3 (tf32).
# ------------------------------------------------------------------------------------------
TC_TOL = {pd.BF16: 2e-2, pd.TF32: 5e-3}
TC_UNIT = {pd.BF16: 2.0 ** -8, pd.TF32: 2.0 ** -10}


def _nrel(got, ref):
    a = np.concatenate([got[k].ravel() for k in ref])
    b = np.concatenate([ref[k].ravel() for k in ref])
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("prec", [pd.BF16, pd.TF32])
@pytest.mark.parametrize("kind,m", [("chain", 40), ("chain", 700), ("cyl", 1000), ("tfim", 300)])
def test_heff_apply_tensor_core(prec, kind, m):
    mpo, qn, bl, br, _, j, rng = _bond_case(kind, m, 4)
    W1, W2 = mpo.W[j], mpo.W[j + 1]
    f0, f1, f2 = mpo.flux[j], mpo.flux[j + 1], mpo.flux[j + 2]
    Lenv = LY.random_env(bl, f0, rng)
    Renv = LY.random_env(br, f2, rng)
    psi = {k: rng.standard_normal((bl[k[0]], br[k[0] + qn[k[1]] + qn[k[2]]])) for k in LY.psi_keys(bl, br, qn)}
    ref = O.heff_apply(Lenv, W1, f0, W2, f2, Renv, psi, qn)
    bond = pd.Bond(qn, bl, br, W1, f0, f1, W2, f2)
    Ld, Rd = _dev(LY.pack_env(Lenv, bl, f0)), _dev(LY.pack_env(Renv, br, f2))
    x = _dev(LY.pack_psi(psi, bl, br, qn))
    y = torch.zeros_like(x)
    pd.heff_apply(bond, prec, Ld.data_ptr(), Rd.data_ptr(), x.data_ptr(), y.data_ptr())
    torch.cuda.synchronize()
    got = LY.unpack_psi(y.cpu().numpy(), bl, br, qn)
    err = _nrel(got, ref)
    assert err <= TC_TOL[prec], err
    assert err > 0.0        # the tensor-core path really ran in reduced precision
    # element-wise: a wrong or mis-scattered block of small norm fails here
    absref = O.heff_apply({k: np.abs(v) for k, v in Lenv.items()}, np.abs(W1), f0, np.abs(W2), f2,
                          {k: np.abs(v) for k, v in Renv.items()}, {k: np.abs(v) for k, v in psi.items()}, qn)
    worst = 0.0
    for k in ref:
        bound = 8.0 * TC_UNIT[prec] * absref[k] + 1e-300
        e = np.abs(got[k] - ref[k])
        worst = max(worst, float((e / bound).max()))
        assert np.all(e <= bound), (k, worst)
    for k in set(got) - set(ref):        # blocks with no contributing term stay exactly zero
        assert not np.any(got[k]), k


@pytest.mark.parametrize("kind,m", [("chain", 500), ("cyl", 800)])
def test_env_updates_tf32(kind, m):
    mpo, qn, bl, _, bm, j, rng = _bond_case(kind, m, 5)
    W = mpo.W[j]
    fL, fR = mpo.flux[j], mpo.flux[j + 1]
    A = {k: rng.standard_normal((bl[k[0]], bm[k[0] + qn[k[1]]])) for k in LY.site_keys(bl, bm, qn)}
    Lin = LY.random_env(bl, fL, rng)
    Rin = LY.random_env(bm, fR, rng)
    bond = pd.Bond(qn, bl, bm, W, fL, fR)
    Lin_d, A_d, Rin_d = _dev(LY.pack_env(Lin, bl, fL)), _dev(LY.pack_site(A, bl, bm, qn)), _dev(LY.pack_env(Rin, bm, fR))
    Lo = torch.zeros(sum(bm[q] * bm[q - int(fR[w])] for q, w in LY.env_keys(bm, fR)), dtype=torch.float64, device="cuda")
    Ro = torch.zeros(sum(bl[q] * bl[q - int(fL[w])] for q, w in LY.env_keys(bl, fL)), dtype=torch.float64, device="cuda")
    pd.env_left(bond, pd.TF32, Lin_d.data_ptr(), A_d.data_ptr(), Lo.data_ptr())
    pd.env_right(bond, pd.TF32, Rin_d.data_ptr(), A_d.data_ptr(), Ro.data_ptr())
    torch.cuda.synchronize()
    refL = O.env_left(Lin, A, W, fL, fR, qn)
    refR = O.env_right(Rin, A, W, fL, fR, qn)
    gotL = LY.unpack_env(Lo.cpu().numpy(), bm, fR)
    gotR = LY.unpack_env(Ro.cpu().numpy(), bl, fL)
    refL = {k: refL.get(k, np.zeros_like(gotL[k])) for k in gotL}
    refR = {k: refR.get(k, np.zeros_like(gotR[k])) for k in gotR}
    # environment updates run at FP32 accuracy in the mixed modes
    assert _nrel(gotL, refL) <= 1e-5
    assert _nrel(gotR, refR) <= 1e-5
