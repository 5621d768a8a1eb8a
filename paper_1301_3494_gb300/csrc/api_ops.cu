// C ABI: operation-level entry points (single steps on caller device buffers).
#include <cstring>
#include <memory>

#include "plans.h"

namespace pd {
thread_local std::string g_last_error;

Sec make_sec(int n, const int* q, const int* m) {
    PD_REQUIRE(n >= 0 && (n == 0 || (q && m)), DMRG_ERR_ARG, "bad sector list");
    Sec s;
    for (int i = 0; i < n; ++i) {
        PD_REQUIRE(m[i] > 0, DMRG_ERR_ARG, "sector dimension must be positive");
        if (i) PD_REQUIRE(q[i] > q[i - 1], DMRG_ERR_ARG, "sector charges must ascend strictly");
        s.q.push_back(q[i]);
        s.m.push_back(m[i]);
    }
    return s;
}

SiteMPO make_site_mpo(int Dl, int Dr, int d, const int* fl, const int* fr, const double* W, const std::vector<int>& qn) {
    PD_REQUIRE(Dl > 0 && Dr > 0 && d > 0 && fl && fr && W, DMRG_ERR_ARG, "bad MPO tensor description");
    SiteMPO s;
    s.Dl = Dl; s.Dr = Dr; s.d = d;
    s.W.assign(W, W + (size_t)Dl * d * d * Dr);
    s.fl.assign(fl, fl + Dl);
    s.fr.assign(fr, fr + Dr);
    for (int w = 0; w < Dl; ++w)
        for (int a = 0; a < d; ++a)
            for (int b = 0; b < d; ++b)
                for (int wp = 0; wp < Dr; ++wp)
                    if (s.at(w, a, b, wp) != 0.0)
                        PD_REQUIRE(qn[a] - qn[b] == s.fr[wp] - s.fl[w], DMRG_ERR_QN,
                                   "MPO element violates the flux rule q(s)-q(s') = f(w')-f(w)");
    return s;
}

dmrg_status fail(const Error& e) {
    g_last_error = e.msg;
    return e.st;
}

void check_err_word(unsigned* err, cudaStream_t st) {
    unsigned h = 0;
    PD_CK(cudaMemcpyAsync(&h, err, 4, cudaMemcpyDeviceToHost, st));
    PD_CK(cudaStreamSynchronize(st));
    if (h & ERRBIT_TIMEOUT) throw Error{DMRG_ERR_TIMEOUT, "a bounded device wait ran out"};
    if (h & ERRBIT_BOUNDS) throw Error{DMRG_ERR_CAPACITY, "a device index check failed"};
    if (h & ERRBIT_NONFINITE) throw Error{DMRG_ERR_NUMERIC, "non-finite value detected"};
}

}  // namespace pd

using namespace pd;

namespace {
struct BondCtx {
    std::vector<int> qn;
    Sec bl, br;
    SiteMPO w1, w2;
};

BondCtx read_bond(const dmrg_bond_desc* bd, bool need_w2) {
    PD_REQUIRE(bd && bd->d > 0 && bd->d <= 8 && bd->qn_local, DMRG_ERR_ARG, "bad bond descriptor");
    BondCtx b;
    b.qn.assign(bd->qn_local, bd->qn_local + bd->d);
    b.bl = make_sec(bd->nl, bd->ql, bd->ml);
    b.br = make_sec(bd->nr, bd->qr, bd->mr);
    b.w1 = make_site_mpo(bd->D0, bd->D1, bd->d, bd->f0, bd->f1, bd->W1, b.qn);
    if (need_w2) b.w2 = make_site_mpo(bd->D1, bd->D2, bd->d, bd->f1, bd->f2, bd->W2, b.qn);
    return b;
}

bool valid_prec(int p) { return p == DMRG_FP64 || p == DMRG_TF32 || p == DMRG_BF16; }
}  // namespace

extern "C" {

const char* dmrg_status_string(int s) {
    switch (s) {
        case DMRG_OK: return "ok";
        case DMRG_ERR_ARG: return "invalid argument";
        case DMRG_ERR_CUDA: return "CUDA error";
        case DMRG_ERR_OOM: return "out of device memory";
        case DMRG_ERR_CAPACITY: return "capacity exceeded";
        case DMRG_ERR_QN: return "quantum-number inconsistency";
        case DMRG_ERR_NUMERIC: return "numerical failure";
        case DMRG_ERR_TIMEOUT: return "bounded device wait ran out";
        case DMRG_ERR_STATE: return "invalid state";
        default: return "unknown status";
    }
}

dmrg_status dmrg_heff_apply(const dmrg_bond_desc* bd, int prec, const double* L_dev, const double* R_dev,
                            const double* x_dev, double* y_dev, double* flops_out, void* stream) {
    try {
        PD_REQUIRE(valid_prec(prec), DMRG_ERR_ARG, "unknown precision");
        PD_REQUIRE(L_dev && R_dev && x_dev && y_dev, DMRG_ERR_ARG, "null buffer");
        cudaStream_t st = (cudaStream_t)stream;
        BondCtx b = read_bond(bd, true);
        TwoSiteMPO t = two_site_mpo(b.w1, b.w2);
        EnvSlab L, R;
        env_alloc(L, b.bl, b.w1.fl, prec, st);
        env_from_packed(L, L_dev, st);
        env_alloc(R, b.br, b.w2.fr, prec, st);
        env_from_packed(R, R_dev, st);
        env_make_operand(L, prec, st);
        env_make_operand(R, prec, st);
        auto plan = make_heff_plan(b.bl, b.br, b.qn, t, L.lay, R.lay, prec, st);
        DBuf err;
        err.ensure(4, st);
        PD_CK(cudaMemsetAsync(err.p, 0, 4, st));
        heff_apply(*plan, L, R, x_dev, y_dev, err.as<unsigned>(), st);
        check_err_word(err.as<unsigned>(), st);
        if (flops_out) *flops_out = plan->flops;
        return DMRG_OK;
    } catch (const Error& e) {
        return fail(e);
    }
}

dmrg_status dmrg_env_left(const dmrg_bond_desc* bd, int prec, const double* Lin_dev, const double* A_dev,
                          double* Lout_dev, void* stream) {
    try {
        PD_REQUIRE(valid_prec(prec), DMRG_ERR_ARG, "unknown precision");
        PD_REQUIRE(Lin_dev && A_dev && Lout_dev, DMRG_ERR_ARG, "null buffer");
        cudaStream_t st = (cudaStream_t)stream;
        BondCtx b = read_bond(bd, false);
        EnvSlab Li, Lo;
        env_alloc(Li, b.bl, b.w1.fl, prec, st);
        env_from_packed(Li, Lin_dev, st);
        env_alloc(Lo, b.br, b.w1.fr, prec, st);
        DBuf err;
        err.ensure(4, st);
        PD_CK(cudaMemsetAsync(err.p, 0, 4, st));
        env_update_left(b.bl, b.br, b.qn, b.w1, Li, A_dev, Lo, prec, err.as<unsigned>(), st);
        check_err_word(err.as<unsigned>(), st);
        env_to_packed(Lo, Lout_dev, st);
        return DMRG_OK;
    } catch (const Error& e) {
        return fail(e);
    }
}

dmrg_status dmrg_env_right(const dmrg_bond_desc* bd, int prec, const double* Rin_dev, const double* B_dev,
                           double* Rout_dev, void* stream) {
    try {
        PD_REQUIRE(valid_prec(prec), DMRG_ERR_ARG, "unknown precision");
        PD_REQUIRE(Rin_dev && B_dev && Rout_dev, DMRG_ERR_ARG, "null buffer");
        cudaStream_t st = (cudaStream_t)stream;
        BondCtx b = read_bond(bd, false);
        EnvSlab Ri, Ro;
        env_alloc(Ri, b.br, b.w1.fr, prec, st);
        env_from_packed(Ri, Rin_dev, st);
        env_alloc(Ro, b.bl, b.w1.fl, prec, st);
        DBuf err;
        err.ensure(4, st);
        PD_CK(cudaMemsetAsync(err.p, 0, 4, st));
        env_update_right(b.bl, b.br, b.qn, b.w1, Ri, B_dev, Ro, prec, err.as<unsigned>(), st);
        check_err_word(err.as<unsigned>(), st);
        env_to_packed(Ro, Rout_dev, st);
        return DMRG_OK;
    } catch (const Error& e) {
        return fail(e);
    }
}

dmrg_status dmrg_svd_split(const dmrg_bond_desc* bd, const double* psi_dev, int m_max, int accurate, double* A_dev,
                           double* lam_dev, double* B_dev, int cap, int* nm_out, int* qm_out, int* mm_out,
                           double* trunc_out, void* stream) {
    try {
        PD_REQUIRE(bd && bd->d > 0 && bd->qn_local, DMRG_ERR_ARG, "bad bond descriptor");
        PD_REQUIRE(psi_dev && A_dev && B_dev && lam_dev && nm_out && qm_out && mm_out, DMRG_ERR_ARG, "null buffer");
        PD_REQUIRE(m_max >= 1, DMRG_ERR_ARG, "m_max must be >= 1");
        cudaStream_t st = (cudaStream_t)stream;
        std::vector<int> qn(bd->qn_local, bd->qn_local + bd->d);
        Sec bl = make_sec(bd->nl, bd->ql, bd->ml), br = make_sec(bd->nr, bd->qr, bd->mr);
        PD_REQUIRE(accurate >= 0 && accurate <= 6 && accurate != 3, DMRG_ERR_ARG, "mode must be 0-2, or 4-6");
        const int plain = accurate >= 4;
        accurate &= 3;
        const bool fp32 = accurate == 2;
        const int saved_qr = g_svd_qr;
        g_svd_qr = plain ? 0 : 1;
        SplitResult r;
        try {
            r = svd_split(bl, br, qn, qn, psi_dev, m_max, 1e-12, accurate == 1, 0, 0, A_dev, B_dev, lam_dev, st, fp32);
        } catch (...) {
            g_svd_qr = saved_qr;
            throw;
        }
        g_svd_qr = saved_qr;
        if (fp32) orthonormalize_factor(bl, r.mid, qn, A_dev, true, st);
        PD_REQUIRE(r.mid.n() <= cap, DMRG_ERR_CAPACITY, "output sector capacity too small");
        *nm_out = r.mid.n();
        for (int i = 0; i < r.mid.n(); ++i) {
            qm_out[i] = r.mid.q[i];
            mm_out[i] = r.mid.m[i];
        }
        if (trunc_out) *trunc_out = r.trunc;
        return DMRG_OK;
    } catch (const Error& e) {
        return fail(e);
    }
}

dmrg_status dmrg_svd_split_batch(int n_bonds, const dmrg_bond_desc* bds, const double* const* psi_devs,
                                 const int* m_max, int mode, double* const* A_devs, double* const* lam_devs,
                                 double* const* B_devs, int cap, int* nm_out, int* qm_out, int* mm_out,
                                 double* trunc_out, void* stream) {
    try {
        PD_REQUIRE(n_bonds >= 0, DMRG_ERR_ARG, "n_bonds must be >= 0");
        if (n_bonds == 0) return DMRG_OK;
        PD_REQUIRE(bds && psi_devs && m_max && A_devs && lam_devs && B_devs && nm_out && qm_out && mm_out,
                   DMRG_ERR_ARG, "null array");
        PD_REQUIRE(mode >= 0 && mode <= 6 && mode != 3, DMRG_ERR_ARG, "mode must be 0-2, or 4-6");
        cudaStream_t st = (cudaStream_t)stream;
        const int plain = mode >= 4;
        const int acc = mode & 3;
        const bool fp32 = acc == 2;
        std::vector<std::vector<int>> qns(n_bonds);
        std::vector<SplitReq> reqs(n_bonds);
        for (int b = 0; b < n_bonds; ++b) {
            const dmrg_bond_desc* bd = bds + b;
            PD_REQUIRE(bd->d > 0 && bd->qn_local, DMRG_ERR_ARG, "bad bond descriptor");
            PD_REQUIRE(psi_devs[b] && A_devs[b] && B_devs[b] && lam_devs[b], DMRG_ERR_ARG, "null buffer");
            PD_REQUIRE(m_max[b] >= 1, DMRG_ERR_ARG, "m_max must be >= 1");
            qns[b].assign(bd->qn_local, bd->qn_local + bd->d);
            SplitReq& r = reqs[b];
            r.bl = make_sec(bd->nl, bd->ql, bd->ml);
            r.br = make_sec(bd->nr, bd->qr, bd->mr);
            r.qn1 = &qns[b];
            r.qn2 = &qns[b];
            r.psi = psi_devs[b];
            r.m_max = m_max[b];
            r.A_out = A_devs[b];
            r.B_out = B_devs[b];
            r.lam_out_dev = lam_devs[b];
        }
        const int saved_qr = g_svd_qr;
        g_svd_qr = plain ? 0 : 1;
        std::vector<SplitResult> res;
        try {
            res = svd_split_batch(reqs, acc == 1, fp32, st);
        } catch (...) {
            g_svd_qr = saved_qr;
            throw;
        }
        g_svd_qr = saved_qr;
        for (int b = 0; b < n_bonds; ++b) {
            const SplitResult& r = res[b];
            if (fp32) orthonormalize_factor(reqs[b].bl, r.mid, qns[b], A_devs[b], true, st);
            PD_REQUIRE(r.mid.n() <= cap, DMRG_ERR_CAPACITY, "output sector capacity too small");
            nm_out[b] = r.mid.n();
            for (int i = 0; i < r.mid.n(); ++i) {
                qm_out[(long long)b * cap + i] = r.mid.q[i];
                mm_out[(long long)b * cap + i] = r.mid.m[i];
            }
            if (trunc_out) trunc_out[b] = r.trunc;
        }
        PD_CK(cudaStreamSynchronize(st));
        return DMRG_OK;
    } catch (const Error& e) {
        return fail(e);
    }
}

dmrg_status dmrg_gemm64(const dmrg_gemm_problem* probs, int n_probs, const dmrg_gemm_segment* segs, int n_segs,
                        const double* A_dev, const double* B_dev, double* C_dev, int mode, int* info, void* stream) {
    try {
        PD_REQUIRE(n_probs >= 0 && n_segs >= 0 && (n_probs == 0 || (probs && segs)), DMRG_ERR_ARG, "bad problem list");
        PD_REQUIRE(mode == 0 || mode == 1, DMRG_ERR_ARG, "mode must be 0 or 1");
        PD_REQUIRE(A_dev && B_dev && C_dev, DMRG_ERR_ARG, "null buffer");
        cudaStream_t st = (cudaStream_t)stream;
        GemmBatch g;
        for (int i = 0; i < n_probs; ++i) {
            const dmrg_gemm_problem& p = probs[i];
            PD_REQUIRE(p.M >= 0 && p.N >= 0 && p.nseg >= 1 && p.seg0 >= 0 && p.seg0 + p.nseg <= n_segs, DMRG_ERR_ARG,
                       "bad problem");
            std::vector<GSeg> sg;
            for (int k = 0; k < p.nseg; ++k) {
                const dmrg_gemm_segment& s = segs[p.seg0 + k];
                PD_REQUIRE(s.K >= 1, DMRG_ERR_ARG, "segment K must be >= 1");
                sg.push_back({s.a_off, s.b_off, s.K, 0});
            }
            g.add(p.M, p.N, p.c_off, p.sam, p.sak, p.sbn, p.sbk, p.scm, p.scn, sg, p.accumulate ? 1 : 0, p.alpha);
        }
        if (info) info[0] = info[1] = info[2] = 0;
        if (g.empty()) return DMRG_OK;       // nothing to compute: no device call
        if (mode == 1) {
            PD_REQUIRE(tc_available(), DMRG_ERR_STATE, "FP64 emulation needs sm_103 tensor cores");
            if (run_gemm64_emu(g, A_dev, B_dev, C_dev, st)) {
                if (info) emu_plan_info(g, info, info + 1, info + 2);
            } else {
                // a plan that exists but was not run: its scale guard sent the batch to the FP64
                // units (info stays 0); no plan: K is too large for exact FP32 accumulation
                int beta = 0, s = 0, groups = 0;
                emu_plan_info(g, &beta, &s, &groups);
                PD_REQUIRE(beta > 0, DMRG_ERR_CAPACITY, "K too large for exact FP32 accumulation");
                const int saved = g_gemm64_emu;
                g_gemm64_emu = 0;
                try {
                    run_gemm64(g, A_dev, B_dev, C_dev, st);
                } catch (...) {
                    g_gemm64_emu = saved;
                    throw;
                }
                g_gemm64_emu = saved;
            }
        } else {
            const int saved = g_gemm64_emu;
            g_gemm64_emu = 0;
            try {
                run_gemm64(g, A_dev, B_dev, C_dev, st);
            } catch (...) {
                g_gemm64_emu = saved;
                throw;
            }
            g_gemm64_emu = saved;
        }
        PD_CK(cudaStreamSynchronize(st));
        return DMRG_OK;
    } catch (const Error& e) {
        return fail(e);
    }
}

}  // extern "C"
