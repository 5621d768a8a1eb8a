"""FP64-accurate grouped GEMM on the bf16 tensor cores (dmrg_gemm64 mode 1) against numpy's FP64
products, and engines running their FP64 GEMMs through it against the FP64-unit engine, the
exact-diagonalisation energy and the oracle's local expectation values."""
import json
import os

import numpy as np
import pytest

import workloads as wl
from oracle import icmps as IC
from tests._gpu import load_mps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

pd = pytest.importorskip("paper_1301_3494_gb300")

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "ed_energies.json")))


class _Batch:
    """Random grouped-GEMM batch in flat host arrays: row-major and transposed operands, operand
    blocks shared between problems, multi-segment problems, accumulation and alpha, rows whose
    magnitudes spread over 2 * spread decades."""

    def __init__(self, rng, nprob, kmax, max_seg, spread, mn_max=300):
        self.A, self.B, self.C0 = [], [], []
        self.na = self.nb = self.nc = 0
        self.probs, self.segs, self.ref = [], [], []
        prev = None
        for _ in range(nprob):
            share = prev is not None and rng.random() < 0.3
            if share:
                # same A blocks as the previous problem (same rows, strides, K), new B blocks
                M, sam, sak, ablocks = prev
                nseg = len(ablocks)
            else:
                M = int(rng.integers(1, mn_max))
                nseg = int(rng.integers(1, max_seg + 1))
                if rng.random() < 0.5:
                    sam, sak = kmax + int(rng.integers(0, 3)), 1
                else:
                    sam, sak = 1, M + int(rng.integers(0, 3))
                rowsA = 10.0 ** rng.uniform(-spread, spread, (M, 1))
                ablocks = []
                for _s in range(nseg):
                    K = int(rng.integers(1, kmax + 1))
                    Am = rng.standard_normal((M, K)) * rowsA
                    ablocks.append((self._put(Am, sam, sak, "A"), Am))
            N = int(rng.integers(1, mn_max))
            if rng.random() < 0.5:
                sbn, sbk = kmax + int(rng.integers(0, 3)), 1
            else:
                sbn, sbk = 1, N + int(rng.integers(0, 3))
            seg0 = len(self.segs)
            acc = np.zeros((M, N))
            for a_off, Am in ablocks:
                K = Am.shape[1]
                Bm = rng.standard_normal((N, K)) * 10.0 ** rng.uniform(-spread, spread, (N, 1))
                b_off = self._put(Bm, sbn, sbk, "B")
                self.segs.append((a_off, b_off, K))
                acc += Am @ Bm.T
            alpha = float(rng.choice([1.0, -0.5, 3.0]))
            accumulate = int(rng.random() < 0.3)
            scm, scn = (1, M) if rng.random() < 0.5 else (N, 1)
            c0 = rng.standard_normal((M, N))
            flat = np.zeros(M * N)
            mm, nn = np.meshgrid(np.arange(M), np.arange(N), indexing="ij")
            flat[mm * scm + nn * scn] = c0
            self.C0.append(flat)
            self.probs.append((M, N, seg0, nseg, self.nc, sam, sak, sbn, sbk, scm, scn, accumulate, alpha))
            self.nc += M * N
            self.ref.append((alpha * acc + (c0 if accumulate else 0.0), ablocks))
            prev = (M, sam, sak, ablocks)

    def _put(self, X, s_row, s_k, side):
        R, K = X.shape
        size = (R - 1) * s_row + (K - 1) * s_k + 1
        buf = np.zeros(size)
        rr, kk = np.meshgrid(np.arange(R), np.arange(K), indexing="ij")
        buf[rr * s_row + kk * s_k] = X
        if side == "A":
            off = self.na
            self.A.append(buf)
            self.na += size
        else:
            off = self.nb
            self.B.append(buf)
            self.nb += size
        return off

    def run(self, mode):
        A = torch.as_tensor(np.concatenate(self.A)).cuda()
        B = torch.as_tensor(np.concatenate(self.B)).cuda()
        C = torch.as_tensor(np.concatenate(self.C0)).cuda()
        info = pd.gemm64(self.probs, self.segs, A.data_ptr(), B.data_ptr(), C.data_ptr(), mode)
        return C.cpu().numpy(), info

    def check(self, Cflat, tol_mult):
        """Error bound per element: tol_mult * K_tot * 2^-53 |alpha| max_k|A(m,:)| max_k|B(n,:)|
        (row maxima over all segments of the problem) plus an ulp of the result."""
        Bf = np.concatenate(self.B)
        worst = 0.0
        for p, (ref, ablocks) in zip(self.probs, self.ref):
            M, N, seg0, nseg, c_off, _sam, _sak, sbn, sbk, scm, scn, _acc, alpha = p
            mm, nn = np.meshgrid(np.arange(M), np.arange(N), indexing="ij")
            got = Cflat[c_off + mm * scm + nn * scn]
            amax, bmax, ktot = np.zeros(M), np.zeros(N), 0
            for s in range(nseg):
                _a_off, b_off, K = self.segs[seg0 + s]
                Am = ablocks[s][1]
                nk, kk = np.meshgrid(np.arange(N), np.arange(K), indexing="ij")
                Bm = Bf[b_off + nk * sbn + kk * sbk]
                amax = np.maximum(amax, np.abs(Am).max(axis=1))
                bmax = np.maximum(bmax, np.abs(Bm).max(axis=1))
                ktot += K
            bound = tol_mult * ktot * 2.0 ** -53 * abs(alpha) * np.outer(amax, bmax) + 2.0 ** -52 * np.abs(ref)
            err = np.abs(got - ref)
            worst = max(worst, float((err / bound).max()))
            assert np.all(err <= bound), worst
        return worst


@pytest.mark.parametrize("case", [(24, 300, 1, 6.0), (12, 700, 3, 4.0), (3, 5000, 1, 2.0), (30, 64, 2, 8.0)])
def test_emulated_gemm_is_fp64_accurate(case):
    nprob, kmax, max_seg, spread = case
    rng = np.random.default_rng(nprob * 7 + kmax)
    b = _Batch(rng, nprob, kmax, max_seg, spread)
    C1, info = b.run(1)
    beta, s, groups = info
    assert 2 <= beta <= 8 and s * beta >= 56 and groups >= s
    b.check(C1, 8.0)
    C0, info0 = b.run(0)
    assert info0 == (0, 0, 0)
    b.check(C0, 8.0)


def test_emulated_gemm_limits():
    # empty batch
    z = torch.zeros(4, dtype=torch.float64, device="cuda")
    assert pd.gemm64([], [], z.data_ptr(), z.data_ptr(), z.data_ptr(), 1) == (0, 0, 0)
    # K beyond exact FP32 accumulation at beta = 2: refused before any device access
    with pytest.raises(pd.DMRGError) as ex:
        pd.gemm64([(1, 1, 0, 1, 0, 1, 1, 1, 1, 1, 1, 0, 1.0)], [(0, 0, 4_000_000)], z.data_ptr(), z.data_ptr(),
                  z.data_ptr(), 1)
    assert ex.value.status == 4


def _engine(mpo, emu, precision="fp64"):
    W, flux, D = wl.pack_mpo(mpo)
    return pd.Engine(W, flux, D, list(mpo.site.qn), mpo.qtot, precision, 8, fp64_emulation=emu)


def test_fp64_engine_with_emulated_gemms():
    """Heisenberg L = 12 (exact at m = 64): the emulated engine follows the FP64-unit engine
    sweep by sweep and reaches the ED energy; 4 regions with merges as well."""
    mpo = wl.heisenberg_chain(12)
    qn = list(mpo.site.qn)
    engs = [_engine(mpo, False), _engine(mpo, True)]
    for e in engs:
        load_mps(e, wl.random_mps(12, qn, 0, 8, seed=3), qn)
    for m in (16, 32, 64, 64):
        r = [e.sweep(m)["energy"] for e in engs]
        assert abs(r[0] - r[1]) <= 1e-10 * abs(r[0])
    assert abs(engs[1].energy() - GOLD["heisenberg_chain_L12_Sz0"]) <= 1e-10 * abs(GOLD["heisenberg_chain_L12_Sz0"])
    for e in engs:
        e.close()
    mpo = wl.heisenberg_chain(24)
    qn = list(mpo.site.qn)
    engs = [_engine(mpo, False), _engine(mpo, True)]
    for e in engs:
        load_mps(e, wl.random_mps(24, qn, 0, 8, seed=4), qn)
        e.setup_regions(4, 2, 32)
    for _ in range(3):
        r = [e.sweep(48)["energy"] for e in engs]
        assert abs(r[0] - r[1]) <= 1e-9 * abs(r[0])
    for e in engs:
        e.close()


def test_emulated_local_expectations_match_oracle():
    mpo = wl.heisenberg_square_cylinder(6, 4)
    qn = list(mpo.site.qn)
    eng = _engine(mpo, True)
    load_mps(eng, wl.random_mps(mpo.L, qn, 0, 90, seed=4), qn)
    bonds, data, _ = eng.state()
    sites, off = [], 0
    for j in range(mpo.L):
        n = sum(bonds[j][q] * bonds[j + 1][q + s] for q in bonds[j] for s in qn if q + s in bonds[j + 1])
        sites.append(wl.unpack_site(data[off: off + n], bonds[j], bonds[j + 1], qn))
        off += n
    psi_o, V_o, _ = IC.inverse_canonical(sites, bonds, qn)
    eng.inverse_canonical()
    st = mpo.site
    Sz, Sp, Sm = st.op("Sz"), st.op("Sp"), st.op("Sm")
    ops1 = [Sz, Sz @ Sz]
    ops2 = [np.kron(Sz, Sz) + 0.5 * (np.kron(Sp, Sm) + np.kron(Sm, Sp)), np.kron(Sp, Sm)]
    e1_o, e2_o = IC.all_expectations(psi_o, V_o, qn, ops1, ops2)
    e1, e2, _ = eng.local_expectations(ops1, ops2)
    assert np.abs(e1 - e1_o).max() <= 1e-12
    assert np.abs(e2 - e2_o).max() <= 1e-12
    eng.close()


def _two_problem_batch(scale_z, nan=False):
    """Two problems of two segments each share the A block X; X meets Y (magnitude 1) in the
    first and Z (magnitude scale_z) in the second, so X's rows share one scale class with both.
    Returns flat A, B, the problem and segment tuples and the exact products."""
    rng = np.random.default_rng(11)
    M, N, K = 40, 30, 70
    X, Y, Z = rng.standard_normal((M, K)), rng.standard_normal((M, K)), rng.standard_normal((M, K)) * scale_z
    if nan:
        Z[3, 5] = np.nan
    Bs = [rng.standard_normal((N, K)) for _ in range(4)]
    A = np.concatenate([X.ravel(), Y.ravel(), Z.ravel()])
    B = np.concatenate([b.ravel() for b in Bs])
    segs = [(0, 0, K), (M * K, N * K, K), (0, 2 * N * K, K), (2 * M * K, 3 * N * K, K)]
    probs = [(M, N, 0, 2, 0, K, 1, K, 1, N, 1, 0, 1.0), (M, N, 2, 2, M * N, K, 1, K, 1, N, 1, 0, 1.0)]
    ref = [X @ Bs[0].T + Y @ Bs[1].T, X @ Bs[2].T + Z @ Bs[3].T]
    bound = [2 * K * 2.0 ** -52 * np.outer(np.maximum(np.abs(X).max(1), np.abs(Y).max(1)),
                                           np.maximum(np.abs(Bs[0]).max(1), np.abs(Bs[1]).max(1)))]
    return A, B, probs, segs, ref, bound


def test_emulated_gemm_shared_block_with_unequal_partners():
    """A block shared by two problems whose other operands differ by 1e10 in magnitude: the first
    problem must still be FP64-accurate relative to its own rows (its scale class is inflated by
    the second problem's rows, so the batch goes to the FP64 units); equal partners stay emulated."""
    for scale_z, emulated in ((1e10, False), (1.0, True)):
        A, B, probs, segs, ref, bound = _two_problem_batch(scale_z)
        Ad, Bd = torch.as_tensor(A).cuda(), torch.as_tensor(B).cuda()
        Cd = torch.zeros(2 * 40 * 30, dtype=torch.float64, device="cuda")
        pd.profile_reset()
        info = pd.gemm64(probs, segs, Ad.data_ptr(), Bd.data_ptr(), Cd.data_ptr(), 1)
        fb = pd.profile_read()["emu_fallbacks"]
        C = Cd.cpu().numpy()
        got0 = C[:1200].reshape(40, 30)
        assert np.all(np.abs(got0 - ref[0]) <= bound[0]), np.abs(got0 - ref[0]).max()
        got1 = C[1200:].reshape(40, 30)
        assert np.allclose(got1, ref[1], rtol=1e-13, atol=1e-13 * np.abs(ref[1]).max())
        assert (info[0] > 0) == emulated and fb == (0 if emulated else 1), (info, fb)


def test_emulated_gemm_propagates_nan():
    A, B, probs, segs, ref, _ = _two_problem_batch(1.0, nan=True)
    Ad, Bd = torch.as_tensor(A).cuda(), torch.as_tensor(B).cuda()
    Cd = torch.zeros(2 * 40 * 30, dtype=torch.float64, device="cuda")
    info = pd.gemm64(probs, segs, Ad.data_ptr(), Bd.data_ptr(), Cd.data_ptr(), 1)
    C = Cd.cpu().numpy()
    assert info == (0, 0, 0)
    assert np.isnan(C[1200:].reshape(40, 30)[3]).all()          # row 3 of the second problem
    assert np.isfinite(C[:1200]).all()
