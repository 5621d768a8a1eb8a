// Stateful two-site DMRG engine behind the context C ABI: serial sweeps (Sec. II) and the
// real-space parallel scheme (Sec. II Eqs. inverse/isvd/merge, Fig. 4) with one CUDA stream
// per region on a single GPU.
#include <chrono>
#include <cmath>
#include <map>
#include <memory>
#include <thread>

#include "plans.h"

namespace pd {
extern thread_local std::string g_last_error;
Sec make_sec(int n, const int* q, const int* m);
SiteMPO make_site_mpo(int Dl, int Dr, int d, const int* fl, const int* fr, const double* W, const std::vector<int>& qn);
void check_err_word(unsigned* err, cudaStream_t st);
}  // namespace pd

using namespace pd;

namespace {

struct StepStats {
    double energy = 0.0, trunc = 0.0, mv_ms = 0.0, mv_flops = 0.0, acc_ms = 0.0;
    int m = 0, matvecs = 0, nonconv = 0, steps = 0, acc_matvecs = 0;
    // merge fidelities 1 - |<Psi'|Psi>| (rounding can take an exact prediction a few ulps below 0,
    // so "none yet" is the count, not a sentinel value)
    double fid_min = -1.0, fid_max = -1.0;
    int nfid = 0;
    void merge(const StepStats& o) {
        trunc = std::max(trunc, o.trunc);
        m = std::max(m, o.m);
        matvecs += o.matvecs;
        nonconv += o.nonconv;
        steps += o.steps;
        mv_ms += o.mv_ms;
        mv_flops += o.mv_flops;
        acc_ms += o.acc_ms;
        acc_matvecs += o.acc_matvecs;
        if (o.nfid > 0) {
            fid_min = nfid ? std::min(fid_min, o.fid_min) : o.fid_min;
            fid_max = nfid ? std::max(fid_max, o.fid_max) : o.fid_max;
            nfid += o.nfid;
        }
    }
};

// One MPS segment: the whole chain (serial mode) or one region.
struct Chain {
    int p = 0, q = 0;                               // sites p..q
    std::vector<Sec> bond;                          // L+1
    std::vector<DBuf> site;                         // L, packed FP64
    std::vector<std::unique_ptr<EnvSlab>> Lenv, Renv;   // L+1
    std::vector<std::vector<double>> lam;           // L+1
    int oc = 0;
    cudaStream_t st = nullptr;
    bool own_stream = false;
    DBuf err;
    StepStats acc;
    void init(int L, cudaStream_t s) {
        bond.assign(L + 1, Sec());
        site.clear();
        site.resize(L);
        Lenv.clear();
        Renv.clear();
        for (int i = 0; i <= L; ++i) {
            Lenv.emplace_back(new EnvSlab());
            Renv.emplace_back(new EnvSlab());
        }
        lam.assign(L + 1, {});
        st = s;
        err.ensure(4, st);
        PD_CK(cudaMemsetAsync(err.p, 0, 4, st));
    }
    void rebind_all() {
        for (auto& b : site) b.rebind(st);
        for (auto& e : Lenv) if (e) e->rebind(st);
        for (auto& e : Renv) if (e) e->rebind(st);
        err.rebind(st);
    }
};

// Streams created by the context; destroyed after every buffer that may free on them.
struct StreamHolder {
    std::vector<cudaStream_t> s;
    ~StreamHolder() {
        for (auto x : s) {
            cudaStreamSynchronize(x);
            cudaStreamDestroy(x);
        }
    }
};

}  // namespace

struct dmrg_ctx {
    StreamHolder streams;                            // first member: destroyed last
    int L = 0, d = 0, qtot = 0;
    std::vector<int> qn;
    std::vector<SiteMPO> W;
    std::vector<std::unique_ptr<TwoSiteMPO>> w12;   // per bond (j, j+1), lazily built
    int prec = DMRG_FP64, kmax = 8;
    bool svd_fp64 = false;       // mixed modes: FP64 splits on ordinary bonds too
    bool emu = false;            // FP64 grouped GEMMs on the bf16 tensor cores (ozaki.cu)
    bool svd_plain = false;      // splits by the plain Jacobi on W (no QR preconditioning)
    bool env64 = false;          // mixed modes: FP64-accurate environments (PREC_ENV64)
    int acc_edges = 0;           // mixed modes: FP64 solves next to region boundaries (2: FP64 splits there too)
    cudaStream_t base = nullptr;
    std::unique_ptr<Chain> serial;
    std::vector<std::unique_ptr<Chain>> reg;
    std::vector<int> bounds;
    std::map<int, std::vector<double>> V;   // boundary bond -> V = 1/lambda (sector order of that bond)
    std::map<int, Sec> Vbond;
    bool have_state = false;
    int dir = 1;                                     // serial sweep direction of dmrg_advance
    std::string last_err;
    std::unique_ptr<ICMPS, void (*)(ICMPS*)> ic{nullptr, icmps_free};   // inverse canonical copy of the state

    const TwoSiteMPO& pair(int j) {
        if (!w12[j]) w12[j].reset(new TwoSiteMPO(two_site_mpo(W[j], W[j + 1])));
        return *w12[j];
    }
};

namespace {

const std::vector<int> kZero1 = {0};

// Arithmetic and storage of the environments: the mixed modes keep them in FP32 unless the
// context asks for FP64-accurate ones.
int eprec(const dmrg_ctx* c) { return (c->env64 && c->prec != DMRG_FP64) ? PREC_ENV64 : c->prec; }

// FP64 local solves (FP64 matvec on the FP64-accurate environments, Davidson to a 1e-10 residual,
// FP64 split) for the bond steps that produce or consume a region's edge tensor next to a
// boundary, and for the merges: the prediction Psi' = psi'_3 V psi'_4 divides the edge tensors by
// the shared bond's singular values, so their errors must sit far below the smallest of them.
bool fp64_solve(const dmrg_ctx* c) { return c->acc_edges > 0 && c->prec != DMRG_FP64; }
bool fp64_edge_split(const dmrg_ctx* c) { return c->acc_edges > 1 && c->prec != DMRG_FP64; }

// FP64 copy of an environment in the same layout (FP32-stored environments of the mixed modes;
// the FP64 solve reads FP64 operands).
const EnvSlab& env64_view(const EnvSlab& e, EnvSlab& tmp, cudaStream_t st) {
    if (e.num == Num::F64) return e;
    tmp.lay = e.lay;
    tmp.num = Num::F64;
    const long long n = std::max<long long>(1, e.lay.rows) * e.lay.ld;
    CopyList cl;
    const long long chunk = 1 << 20;
    for (long long s0 = 0; s0 < n; s0 += chunk) {
        CopyJob j{};
        j.src = s0; j.dst = s0; j.rows = 1; j.cols = (int)std::min(chunk, n - s0);
        j.srs = 0; j.scs = 1; j.drs = 0; j.dcs = 1; j.zero_to = 0; j.scale = 1.0;
        cl.add(j);
    }
    cl.up(st);
    tmp.buf.ensure(n * 8, st);
    run_copy<float>(cl, e.buf.as<float>(), tmp.buf.p, Num::F64, st);
    tmp.valid = true;
    return tmp;
}
constexpr double kEdgeTol = 1e-10;
int edge_iters(const dmrg_sweep_params* p) { return std::max(12, p->dav_max_iter + p->refine_iters); }

// ------------------------------------------------------------------------------------------
// Building blocks on a chain
// ------------------------------------------------------------------------------------------
void make_boundary_envs(dmrg_ctx* c, Chain& ch) {
    env_boundary(*ch.Lenv[0], ch.bond[0], c->W[0].fl, eprec(c), ch.st);
    env_boundary(*ch.Renv[c->L], ch.bond[c->L], c->W[c->L - 1].fr, eprec(c), ch.st);
}

// Untruncated right-canonicalisation with the centre on site 0 (SVDs from the right).
void right_canonicalize(dmrg_ctx* c, Chain& ch) {
    const int L = c->L;
    cudaStream_t st = ch.st;
    for (int j = L - 1; j >= 1; --j) {
        const Sec bl = ch.bond[j], br = ch.bond[j + 1];
        long long na, nb, nl;
        svd_split_bounds(bl, br, kZero1, c->qn, &na, &nb, &nl);
        DBuf U, B;
        U.ensure(std::max<long long>(1, na) * 8, st);
        B.ensure(std::max<long long>(1, nb) * 8, st);
        // site j viewed as a two-leg object (trivial first leg): A = U Lambda, B = V^T
        SplitResult r = svd_split(bl, br, kZero1, c->qn, ch.site[j].as<double>(), 1 << 30, 0.0, false, 1, 0,
                                  U.as<double>(), B.as<double>(), nullptr, st);
        // absorb the carry U Lambda into site j-1: new[(x, s)] = old[(x, s)] carry[q]
        const Sec& bp = ch.bond[j - 1];
        const SiteLayout Sold = site_layout(bp, bl, c->qn);
        const SiteLayout Snew = site_layout(bp, r.mid, c->qn);
        const SiteLayout Sc = site_layout(bl, r.mid, kZero1);
        GemmBatch g;
        for (const auto& nbk : Snew.blk) {
            int ob = Sold.at(nbk.i, nbk.s);
            int qa = bp.q[nbk.i] + c->qn[nbk.s];
            int ia = bl.find(qa);
            int cb = Sc.at(ia, 0);
            if (ob < 0 || cb < 0) continue;
            // C(m = k, n = a_x) = sum_old carry[old][k] site[a_x][old]
            g.add(nbk.cols, nbk.rows, nbk.off, 1, nbk.cols, bl.m[ia], 1, 1, nbk.cols,
                  {GSeg{Sc.blk[cb].off, Sold.blk[ob].off, bl.m[ia], 0}});
        }
        DBuf nsite;
        nsite.ensure(std::max<long long>(1, Snew.size) * 8, st);
        PD_CK(cudaMemsetAsync(nsite.p, 0, std::max<long long>(1, Snew.size) * 8, st));
        run_gemm64(g, U.as<double>(), ch.site[j - 1].as<double>(), nsite.as<double>(), st);
        PD_CK(cudaStreamSynchronize(st));
        ch.site[j] = std::move(B);
        ch.site[j - 1] = std::move(nsite);
        ch.bond[j] = r.mid;
    }
    const SiteLayout S0 = site_layout(ch.bond[0], ch.bond[1], c->qn);
    double nn = dot_host(ch.site[0].as<double>(), ch.site[0].as<double>(), S0.size, st);
    PD_REQUIRE(nn > 0 && std::isfinite(nn), DMRG_ERR_NUMERIC, "zero or non-finite initial state");
    scale_vec(ch.site[0].as<double>(), S0.size, 1.0 / std::sqrt(nn), st);
    ch.oc = 0;
}

void build_right_envs(dmrg_ctx* c, Chain& ch, int down_to) {
    for (int j = c->L - 1; j >= down_to; --j) {
        env_alloc(*ch.Renv[j], ch.bond[j], c->W[j].fl, eprec(c), ch.st);
        env_update_right(ch.bond[j], ch.bond[j + 1], c->qn, c->W[j], *ch.Renv[j + 1], ch.site[j].as<double>(),
                         *ch.Renv[j], eprec(c), ch.err.as<unsigned>(), ch.st);
    }
}

// Davidson on psi at bond j (sites j, j+1) with the chain's environments L[j], R[j+2].
DavResult solve_bond(dmrg_ctx* c, Chain& ch, int j, EnvSlab& Lj, EnvSlab& Rj, DBuf& psi, const dmrg_sweep_params* p,
                     StepStats& s, double* flops_per_mv, bool edge = false) {
    if (edge && fp64_solve(c)) {
        EnvSlab l64, r64;
        const EnvSlab& L = env64_view(Lj, l64, ch.st);
        const EnvSlab& R = env64_view(Rj, r64, ch.st);
        auto plan = make_heff_plan(ch.bond[j], ch.bond[j + 2], c->qn, c->pair(j), L.lay, R.lay, DMRG_FP64, ch.st);
        DavResult r = davidson(*plan, L, R, psi.as<double>(), c->kmax, kEdgeTol, edge_iters(p),
                               ch.err.as<unsigned>(), ch.st);
        s.acc_matvecs += r.matvecs;
        s.acc_ms += r.mv_ms;
        if (r.rnorm > kEdgeTol * std::max(1.0, std::fabs(r.theta))) s.nonconv++;
        if (flops_per_mv) *flops_per_mv = plan->flops;
        return r;
    }
    env_make_operand(Lj, c->prec, ch.st);
    env_make_operand(Rj, c->prec, ch.st);
    auto plan = make_heff_plan(ch.bond[j], ch.bond[j + 2], c->qn, c->pair(j), Lj.lay, Rj.lay, c->prec, ch.st);
    std::unique_ptr<HeffPlan> acc;
    if (c->prec != DMRG_FP64 && p->refine_iters > 0) {
        env_make_operand(Lj, PREC_F32, ch.st);
        env_make_operand(Rj, PREC_F32, ch.st);
        acc = make_heff_plan(ch.bond[j], ch.bond[j + 2], c->qn, c->pair(j), Lj.lay, Rj.lay, PREC_F32, ch.st);
    }
    DavResult r = davidson(*plan, Lj, Rj, psi.as<double>(), c->kmax, p->dav_tol, p->dav_max_iter,
                           ch.err.as<unsigned>(), ch.st, acc.get(), p->refine_iters);
    Lj.drop_operands();
    Rj.drop_operands();
    s.matvecs += r.matvecs;
    s.mv_ms += r.mv_ms;
    s.acc_matvecs += r.acc_matvecs;
    s.acc_ms += r.acc_ms;
    s.mv_flops += plan->flops * r.matvecs;
    if (r.rnorm > p->dav_tol * std::max(1.0, std::fabs(r.theta))) s.nonconv++;
    if (flops_per_mv) *flops_per_mv = plan->flops;
    return r;
}

// Mixed-precision modes split ordinary bonds by the FP32 Jacobi; FP64 at shared (accurate) bonds,
// on edge bonds when the context asks for FP64 edge splits, and everywhere in FP64 mode.
bool split_fp32(const dmrg_ctx* c, bool accurate, bool edge) {
    return c->prec != DMRG_FP64 && !accurate && !c->svd_fp64 && !(edge && fp64_edge_split(c));
}

// Output buffers of the split at bond j (FP64, packed A and B blocks).
void alloc_split(dmrg_ctx* c, const Chain& ch, int j, DBuf& A, DBuf& B) {
    long long na, nb, nl;
    svd_split_bounds(ch.bond[j], ch.bond[j + 2], c->qn, c->qn, &na, &nb, &nl);
    A.ensure(std::max<long long>(1, na) * 8, ch.st);
    B.ensure(std::max<long long>(1, nb) * 8, ch.st);
}

// After the split r of psi at bond j into A, B: store A/B/Lambda in the chain and update the
// environment behind the move.
void finish_move(dmrg_ctx* c, Chain& ch, int j, bool right, DBuf& psi, int m_max, bool accurate, bool fp32,
                 SplitResult& r, DBuf& A, DBuf& B, StepStats& s) {
    cudaStream_t st = ch.st;
    const Sec bl = ch.bond[j], br = ch.bond[j + 2];
    if (fp32) {
        // the factor that joins a block must be orthonormal to FP64 accuracy; an FP32 split whose
        // kept vectors are beyond the reach of the re-orthonormalisation (FP32 rounding left
        // near-cutoff columns coupled) is redone in FP64
        bool ok = true;
        try {
            if (right) orthonormalize_factor(bl, r.mid, c->qn, A.as<double>(), true, st);
            else orthonormalize_factor(r.mid, br, c->qn, B.as<double>(), false, st);
        } catch (const Error& e) {
            if (e.st != DMRG_ERR_NUMERIC) throw;
            ok = false;
        }
        if (!ok) {
            prof_fallback();
            r = svd_split(bl, br, c->qn, c->qn, psi.as<double>(), m_max, 1e-12, accurate, right ? 0 : 1,
                          right ? 1 : 0, A.as<double>(), B.as<double>(), nullptr, st, false);
        }
    }
    ch.bond[j + 1] = r.mid;
    ch.lam[j + 1] = r.lam;
    s.trunc = std::max(s.trunc, r.trunc);
    s.m = std::max(s.m, (int)r.mid.total());
    if (right) {
        env_alloc(*ch.Lenv[j + 1], r.mid, c->W[j].fr, eprec(c), st);
        env_update_left(bl, r.mid, c->qn, c->W[j], *ch.Lenv[j], A.as<double>(), *ch.Lenv[j + 1], eprec(c),
                        ch.err.as<unsigned>(), st);
        ch.oc = j + 1;
        // R[j+1] belongs to the bond left of the new centre's two-site window and is rebuilt
        // before it is read again (R[j+2] stays: a step back at bond j reads it)
        if (j + 1 <= ch.q) ch.Renv[j + 1]->release();
    } else {
        env_alloc(*ch.Renv[j + 1], r.mid, c->W[j + 1].fl, eprec(c), st);
        env_update_right(r.mid, br, c->qn, c->W[j + 1], *ch.Renv[j + 2], B.as<double>(), *ch.Renv[j + 1], eprec(c),
                         ch.err.as<unsigned>(), st);
        ch.oc = j;
        // L[j+1] likewise (L[j] stays); the chain's outer environments (L[p], R[q+1]) are kept
        if (j + 1 > ch.p) ch.Lenv[j + 1]->release();
    }
    ch.site[j] = std::move(A);
    ch.site[j + 1] = std::move(B);
}

// Split psi at bond j, store A/B/Lambda in the chain, update the environment behind the move.
void split_and_move(dmrg_ctx* c, Chain& ch, int j, bool right, DBuf& psi, int m_max, bool accurate, StepStats& s,
                    SplitResult* out = nullptr, bool edge = false) {
    DBuf A, B;
    alloc_split(c, ch, j, A, B);
    const bool fp32 = split_fp32(c, accurate, edge);
    SplitResult r = svd_split(ch.bond[j], ch.bond[j + 2], c->qn, c->qn, psi.as<double>(), m_max, 1e-12, accurate,
                              right ? 0 : 1, right ? 1 : 0, A.as<double>(), B.as<double>(), nullptr, ch.st, fp32);
    finish_move(c, ch, j, right, psi, m_max, accurate, fp32, r, A, B, s);
    if (out) *out = r;
}

void form_psi(dmrg_ctx* c, Chain& ch, int j, DBuf& psi) {
    const PsiLayout P = psi_layout(ch.bond[j], ch.bond[j + 2], c->qn);
    psi.ensure(std::max<long long>(1, P.size) * 8, ch.st);
    form_two_site(ch.bond[j], ch.bond[j + 1], ch.bond[j + 2], c->qn, ch.site[j].as<double>(),
                  ch.site[j + 1].as<double>(), nullptr, psi.as<double>(), ch.st);
}

// One two-site DMRG step at bond j (Sec. II): form Psi, Davidson, SVD + truncation, gauge move,
// projected-operator update.
void bond_step(dmrg_ctx* c, Chain& ch, int j, bool right, const dmrg_sweep_params* p, bool accurate = false,
               bool edge = false) {
    PD_REQUIRE(ch.oc == (right ? j : j + 1), DMRG_ERR_STATE, "orthogonality centre not at the bond");
    DBuf psi;
    form_psi(c, ch, j, psi);
    StepStats& s = ch.acc;
    DavResult r = solve_bond(c, ch, j, *ch.Lenv[j], *ch.Renv[j + 2], psi, p, s, nullptr, edge);
    s.energy = r.theta;
    s.steps++;
    split_and_move(c, ch, j, right, psi, p->m_max, accurate, s, nullptr, edge);
}

// Move the centre across bond j by an untruncated SVD (no Davidson).
void gauge_step(dmrg_ctx* c, Chain& ch, int j, bool right) {
    DBuf psi;
    form_psi(c, ch, j, psi);
    StepStats dummy;
    split_and_move(c, ch, j, right, psi, 1 << 30, false, dummy);
}

void copy_site(DBuf& dst, const DBuf& src, long long elems, cudaStream_t st) {
    dst.ensure(std::max<long long>(1, elems) * 8, st);
    if (elems > 0) PD_CK(cudaMemcpyAsync(dst.p, src.p, elems * 8, cudaMemcpyDeviceToDevice, st));
}

void copy_env(EnvSlab& dst, const EnvSlab& src, cudaStream_t st) {
    dst.lay = src.lay;
    dst.num = src.num;
    size_t bytes = (size_t)std::max<long long>(1, src.lay.rows) * src.lay.ld * num_size(src.num);
    dst.buf.ensure(bytes, st);
    PD_CK(cudaMemcpyAsync(dst.buf.p, src.buf.p, bytes, cudaMemcpyDeviceToDevice, st));
    dst.op_valid = false;
    dst.op32_valid = false;
    dst.valid = src.valid;
}

double rayleigh_fp64(dmrg_ctx* c, Chain& ch, int j, const double* psi) {
    // FP64 <psi|H|psi>/<psi|psi> at bond j; in mixed mode with FP64 copies of the FP32 environments
    cudaStream_t st = ch.st;
    EnvSlab L64, R64;
    const EnvSlab* Lp = ch.Lenv[j].get();
    const EnvSlab* Rp = ch.Renv[j + 2].get();
    if (c->prec != DMRG_FP64) {
        env_alloc(L64, ch.bond[j], c->W[j].fl, DMRG_FP64, st);
        env_alloc(R64, ch.bond[j + 2], c->W[j + 1].fr, DMRG_FP64, st);
        DBuf tmp;
        tmp.ensure(std::max<long long>(1, Lp->lay.packed_size) * 8, st);
        env_to_packed(*Lp, tmp.as<double>(), st);
        env_from_packed(L64, tmp.as<double>(), st);
        tmp.ensure(std::max<long long>(1, Rp->lay.packed_size) * 8, st);
        env_to_packed(*Rp, tmp.as<double>(), st);
        env_from_packed(R64, tmp.as<double>(), st);
        PD_CK(cudaStreamSynchronize(st));
        Lp = &L64;
        Rp = &R64;
    }
    auto plan = make_heff_plan(ch.bond[j], ch.bond[j + 2], c->qn, c->pair(j), Lp->lay, Rp->lay, DMRG_FP64, st);
    DBuf y;
    y.ensure(std::max<long long>(1, plan->psi.size) * 8, st);
    heff_apply(*plan, *Lp, *Rp, psi, y.as<double>(), ch.err.as<unsigned>(), st);
    double num = dot_host(psi, y.as<double>(), plan->psi.size, st);
    double den = dot_host(psi, psi, plan->psi.size, st);
    return num / den;
}

// ------------------------------------------------------------------------------------------
// Regions
// ------------------------------------------------------------------------------------------
// Edge bonds of a region: (q-1, q) when bond q+1 is a boundary, (p, p+1) when bond p is one.
bool edge_bond(const dmrg_ctx* c, const Chain& r, int j) {
    return (j == r.q - 1 && r.q + 1 < c->L) || (j == r.p && r.p > 0);
}

void region_half_sweep(dmrg_ctx* c, Chain& r, bool right, const dmrg_sweep_params* p) {
    auto edge = [&](int j) { return edge_bond(c, r, j); };
    if (right) {
        PD_REQUIRE(r.oc == r.p, DMRG_ERR_STATE, "region centre not at its left end");
        for (int j = r.p; j < r.q; ++j) bond_step(c, r, j, true, p, false, edge(j));
    } else {
        PD_REQUIRE(r.oc == r.q, DMRG_ERR_STATE, "region centre not at its right end");
        for (int j = r.q - 1; j >= r.p; --j) bond_step(c, r, j, false, p, false, edge(j));
    }
}

void stream_after(cudaStream_t waiter, cudaStream_t producer);

// Half sweeps of the regions ks (directions right[i]) in lockstep: at step t every region forms
// Psi on its t-th bond and solves it, then the splits of all these bonds run as one batch per
// precision on the context's base stream -- one Jacobi launch over the charge sectors of every
// region's bond, which keeps the SMs busy in the late rounds where one bond's largest sectors
// alone leave most of them idle -- and every region then finishes its own move.
void lockstep_half(dmrg_ctx* c, const std::vector<int>& ks, const std::vector<char>& right,
                   const dmrg_sweep_params* p) {
    const int n = (int)ks.size();
    int steps = 0;
    for (int i = 0; i < n; ++i) {
        const Chain& r = *c->reg[ks[i]];
        PD_REQUIRE(r.oc == (right[i] ? r.p : r.q), DMRG_ERR_STATE, "region centre not at the start of its half sweep");
        steps = std::max(steps, r.q - r.p);
    }
    for (int t = 0; t < steps; ++t) {
        std::vector<DBuf> psi(n), A(n), B(n);
        std::vector<int> js(n, -1);
        std::vector<char> f32(n, 0);
        for (int i = 0; i < n; ++i) {
            Chain& r = *c->reg[ks[i]];
            if (t >= r.q - r.p) continue;
            const int j = right[i] ? r.p + t : r.q - 1 - t;
            const bool edge = edge_bond(c, r, j);
            js[i] = j;
            form_psi(c, r, j, psi[i]);
            StepStats& s = r.acc;
            DavResult d = solve_bond(c, r, j, *r.Lenv[j], *r.Renv[j + 2], psi[i], p, s, nullptr, edge);
            s.energy = d.theta;
            s.steps++;
            f32[i] = split_fp32(c, false, edge);
        }
        // one batch per split precision (FP32 block Jacobi; FP64 for edge bonds when asked for)
        std::vector<SplitResult> res(n);
        for (int prec32 = 1; prec32 >= 0; --prec32) {
            std::vector<SplitReq> reqs;
            std::vector<int> who;
            for (int i = 0; i < n; ++i) {
                if (js[i] < 0 || f32[i] != prec32) continue;
                Chain& r = *c->reg[ks[i]];
                const int j = js[i];
                alloc_split(c, r, j, A[i], B[i]);
                SplitReq q;
                q.bl = r.bond[j];
                q.br = r.bond[j + 2];
                q.qn1 = &c->qn;
                q.qn2 = &c->qn;
                q.psi = psi[i].as<double>();
                q.m_max = p->m_max;
                q.lam_pow_left = right[i] ? 0 : 1;
                q.lam_pow_right = right[i] ? 1 : 0;
                q.A_out = A[i].as<double>();
                q.B_out = B[i].as<double>();
                reqs.push_back(q);
                who.push_back(i);
                stream_after(c->base, r.st);
            }
            if (reqs.empty()) continue;
            std::vector<SplitResult> rb = svd_split_batch(reqs, false, prec32 != 0, c->base);
            for (size_t q = 0; q < who.size(); ++q) {
                res[who[q]] = std::move(rb[q]);
                stream_after(c->reg[ks[who[q]]]->st, c->base);
            }
        }
        for (int i = 0; i < n; ++i) {
            if (js[i] < 0) continue;
            Chain& r = *c->reg[ks[i]];
            finish_move(c, r, js[i], right[i] != 0, psi[i], p->m_max, false, f32[i] != 0, res[i], A[i], B[i], r.acc);
        }
    }
    for (int k : ks) check_err_word(c->reg[k]->err.as<unsigned>(), c->reg[k]->st);
}

// Run fn(i) for i in items on one host thread each (every region drives its own stream).
template <class F>
void parallel_items(const std::vector<int>& items, F fn, bool serial = false) {
    if (serial || items.size() <= 1) {
        // on the calling thread, one after another (each item has the GPU to itself)
        for (int it : items) fn(it);
        return;
    }
    std::vector<std::thread> th;
    std::vector<Error> errs(items.size(), Error{DMRG_OK, ""});
    int dev = 0, sms = 0;
    PD_CK(cudaGetDevice(&dev));
    PD_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int cap = items.size() > 1 ? std::max(1, sms / (int)items.size()) : 0;
    const int emu = g_gemm64_emu, qr = g_svd_qr;
    for (size_t t = 0; t < items.size(); ++t)
        th.emplace_back([&, t]() {
            try {
                PD_CK(cudaSetDevice(dev));
                g_sm_cap = cap;
                g_gemm64_emu = emu;
                g_svd_qr = qr;
                fn(items[t]);
            } catch (const Error& e) {
                errs[t] = e;
            } catch (const std::exception& e) {
                errs[t] = Error{DMRG_ERR_STATE, e.what()};
            }
        });
    for (auto& x : th) x.join();
    for (auto& e : errs)
        if (e.st != DMRG_OK) throw e;
}

void stream_after(cudaStream_t waiter, cudaStream_t producer) {
    if (waiter == producer) return;
    cudaEvent_t ev;
    PD_CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    PD_CK(cudaEventRecord(ev, producer));
    PD_CK(cudaStreamWaitEvent(waiter, ev, 0));
    PD_CK(cudaEventDestroy(ev));
}

// Merge at boundary k between regions k-1 and k: Psi' = psi'_3 V psi'_4 (Eq. merge), Davidson on
// the shared bond with the left region's L and the right region's R environment, accurate SVD,
// new split psi_3 = A Lambda, psi_4 = Lambda B, V = 1/Lambda (Eqs. inverse, isvd), and the
// environment hand-off.
void do_merge(dmrg_ctx* c, int k, const dmrg_sweep_params* p, double* fid_out, double* e_out) {
    Chain& left = *c->reg[k - 1];
    Chain& right = *c->reg[k];
    const int b = c->bounds[k];
    PD_REQUIRE(left.oc == b - 1 && right.oc == b, DMRG_ERR_STATE, "regions are not both at the shared bond");
    cudaStream_t st = left.st;
    stream_after(st, right.st);
    const Sec bm = c->Vbond.at(b);
    PD_REQUIRE(left.bond[b] == bm && right.bond[b] == bm, DMRG_ERR_STATE, "boundary bond changed since the split");
    const Sec bl = left.bond[b - 1], br = right.bond[b + 1];
    DBuf Vd;
    upload(Vd, c->V.at(b), st);
    const PsiLayout P = psi_layout(bl, br, c->qn);
    DBuf psi;
    psi.ensure(std::max<long long>(1, P.size) * 8, st);
    form_two_site(bl, bm, br, c->qn, left.site[b - 1].as<double>(), right.site[b].as<double>(), Vd.as<double>(),
                  psi.as<double>(), st);
    double nn = dot_host(psi.as<double>(), psi.as<double>(), P.size, st);
    PD_REQUIRE(nn > 0 && std::isfinite(nn), DMRG_ERR_NUMERIC, "merged wavefunction is zero or non-finite");
    scale_vec(psi.as<double>(), P.size, 1.0 / std::sqrt(nn), st);
    DBuf guess;
    copy_site(guess, psi, P.size, st);
    EnvSlab& Lj = *left.Lenv[b - 1];
    EnvSlab& Rj = *right.Renv[b + 1];
    StepStats& s = left.acc;
    DavResult r;
    if (fp64_solve(c)) {
        EnvSlab l64, r64;
        const EnvSlab& L = env64_view(Lj, l64, st);
        const EnvSlab& R = env64_view(Rj, r64, st);
        auto plan = make_heff_plan(bl, br, c->qn, c->pair(b - 1), L.lay, R.lay, DMRG_FP64, st);
        r = davidson(*plan, L, R, psi.as<double>(), c->kmax, kEdgeTol, edge_iters(p), left.err.as<unsigned>(), st);
        s.acc_matvecs += r.matvecs;
        s.acc_ms += r.mv_ms;
        if (r.rnorm > kEdgeTol * std::max(1.0, std::fabs(r.theta))) s.nonconv++;
    } else {
        env_make_operand(Lj, c->prec, st);
        env_make_operand(Rj, c->prec, st);
        auto plan = make_heff_plan(bl, br, c->qn, c->pair(b - 1), Lj.lay, Rj.lay, c->prec, st);
        std::unique_ptr<HeffPlan> accp;
        if (c->prec != DMRG_FP64 && p->refine_iters > 0) {
            env_make_operand(Lj, PREC_F32, st);
            env_make_operand(Rj, PREC_F32, st);
            accp = make_heff_plan(bl, br, c->qn, c->pair(b - 1), Lj.lay, Rj.lay, PREC_F32, st);
        }
        r = davidson(*plan, Lj, Rj, psi.as<double>(), c->kmax, p->dav_tol, p->dav_max_iter, left.err.as<unsigned>(),
                     st, accp.get(), p->refine_iters);
        Lj.drop_operands();
        Rj.drop_operands();
        s.matvecs += r.matvecs;
        s.mv_ms += r.mv_ms;
        s.acc_matvecs += r.acc_matvecs;
        s.acc_ms += r.acc_ms;
        s.mv_flops += plan->flops * r.matvecs;
        if (r.rnorm > p->dav_tol * std::max(1.0, std::fabs(r.theta))) s.nonconv++;
    }
    double ov = dot_host(guess.as<double>(), psi.as<double>(), P.size, st);
    double fid = 1.0 - std::fabs(ov);
    s.energy = r.theta;
    s.steps++;
    s.fid_min = s.nfid ? std::min(s.fid_min, fid) : fid;
    s.fid_max = s.nfid ? std::max(s.fid_max, fid) : fid;
    s.nfid++;
    long long na, nb, nl;
    svd_split_bounds(bl, br, c->qn, c->qn, &na, &nb, &nl);
    DBuf A, B;
    A.ensure(std::max<long long>(1, na) * 8, st);
    B.ensure(std::max<long long>(1, nb) * 8, st);
    SplitResult sr = svd_split(bl, br, c->qn, c->qn, psi.as<double>(), p->m_max, 1e-12, true, 0, 0, A.as<double>(),
                               B.as<double>(), nullptr, st);
    s.trunc = std::max(s.trunc, sr.trunc);
    s.m = std::max(s.m, (int)sr.mid.total());
    DBuf lamd;
    upload(lamd, sr.lam, st);
    // new projected operators for both sides (Sec. II: each side's operators in its own basis)
    std::unique_ptr<EnvSlab> Lnew(new EnvSlab()), Rnew(new EnvSlab());
    env_alloc(*Lnew, sr.mid, c->W[b - 1].fr, eprec(c), st);
    env_update_left(bl, sr.mid, c->qn, c->W[b - 1], Lj, A.as<double>(), *Lnew, eprec(c), left.err.as<unsigned>(), st);
    env_alloc(*Rnew, sr.mid, c->W[b].fl, eprec(c), st);
    env_update_right(sr.mid, br, c->qn, c->W[b], Rj, B.as<double>(), *Rnew, eprec(c), left.err.as<unsigned>(), st);
    // psi_3 = A Lambda for the left region, psi_4 = Lambda B for the right region
    const SiteLayout SA = site_layout(bl, sr.mid, c->qn), SB = site_layout(sr.mid, br, c->qn);
    DBuf psi3, psi4;
    psi3.ensure(std::max<long long>(1, SA.size) * 8, st);
    psi4.ensure(std::max<long long>(1, SB.size) * 8, st);
    scale_site(bl, sr.mid, c->qn, A.as<double>(), lamd.as<double>(), true, psi3.as<double>(), st);
    scale_site(sr.mid, br, c->qn, B.as<double>(), lamd.as<double>(), false, psi4.as<double>(), st);
    check_err_word(left.err.as<unsigned>(), st);
    std::vector<double> V(sr.lam.size());
    for (size_t i = 0; i < V.size(); ++i) V[i] = 1.0 / sr.lam[i];
    c->V.at(b) = V;            // keys exist since set-up: lookups only, safe across region threads
    c->Vbond.at(b) = sr.mid;
    left.bond[b] = sr.mid;
    right.bond[b] = sr.mid;
    left.lam[b] = sr.lam;
    right.lam[b] = sr.lam;
    PD_CK(cudaStreamSynchronize(st));
    psi4.rebind(right.st);
    Lnew->rebind(right.st);
    left.site[b - 1] = std::move(psi3);
    right.site[b] = std::move(psi4);
    left.Renv[b] = std::move(Rnew);
    right.Lenv[b] = std::move(Lnew);
    stream_after(right.st, st);
    if (fid_out) *fid_out = fid;
    if (e_out) *e_out = r.theta;
}

// Serial set-up of the regions (warm-up, split at every boundary while sweeping left,
// staggered positions).
void setup_regions(dmrg_ctx* c, int R, int warmup, const dmrg_sweep_params* p) {
    Chain& ch = *c->serial;
    const int L = c->L;
    PD_REQUIRE(ch.oc == 0, DMRG_ERR_STATE, "set-up needs the serial centre on site 0");
    std::vector<int> bounds(R + 1);
    for (int k = 0; k <= R; ++k) bounds[k] = (int)std::lround((double)k * L / R);
    for (int k = 0; k < R; ++k)
        PD_REQUIRE(bounds[k + 1] - bounds[k] >= 2, DMRG_ERR_ARG, "every region needs at least two sites");
    for (int j = 0; j + 1 < L; ++j) c->pair(j);   // build shared read-only data before threads start
    for (int w = 0; w + 1 < warmup; ++w) {
        for (int j = 0; j <= L - 2; ++j) bond_step(c, ch, j, true, p);
        for (int j = L - 2; j >= 0; --j) bond_step(c, ch, j, false, p);
    }
    for (int j = 0; j <= L - 2; ++j) {
        if (warmup > 0) bond_step(c, ch, j, true, p);
        else gauge_step(c, ch, j, true);
    }
    std::map<int, int> bidx;
    for (int k = 1; k < R; ++k) bidx[bounds[k]] = k;
    std::vector<DBuf> left_end(R);
    std::vector<std::unique_ptr<EnvSlab>> left_env(R);
    cudaStream_t st = ch.st;
    for (int j = L - 2; j >= 0; --j) {
        const int b = j + 1;
        const bool split = bidx.count(b) > 0;
        if (!split) {
            if (warmup > 0) bond_step(c, ch, j, false, p);
            else gauge_step(c, ch, j, false);
            continue;
        }
        DBuf psi;
        form_psi(c, ch, j, psi);
        StepStats& s = ch.acc;
        int m_max = warmup > 0 ? p->m_max : (1 << 30);
        if (warmup > 0) {
            DavResult r = solve_bond(c, ch, j, *ch.Lenv[j], *ch.Renv[j + 2], psi, p, s, nullptr);
            s.energy = r.theta;
            s.steps++;
        }
        const Sec bl = ch.bond[j], br = ch.bond[j + 2];
        long long na, nb, nl;
        svd_split_bounds(bl, br, c->qn, c->qn, &na, &nb, &nl);
        DBuf A, B;
        A.ensure(std::max<long long>(1, na) * 8, st);
        B.ensure(std::max<long long>(1, nb) * 8, st);
        SplitResult sr = svd_split(bl, br, c->qn, c->qn, psi.as<double>(), m_max, 1e-12, warmup > 0, 0, 0,
                                   A.as<double>(), B.as<double>(), nullptr, st);
        DBuf lamd;
        upload(lamd, sr.lam, st);
        const int k = bidx[b];
        // region k: left-end centre Lambda B and its left environment built from A
        const SiteLayout SA = site_layout(bl, sr.mid, c->qn), SB = site_layout(sr.mid, br, c->qn);
        left_end[k].ensure(std::max<long long>(1, SB.size) * 8, st);
        scale_site(sr.mid, br, c->qn, B.as<double>(), lamd.as<double>(), false, left_end[k].as<double>(), st);
        left_env[k].reset(new EnvSlab());
        env_alloc(*left_env[k], sr.mid, c->W[j].fr, eprec(c), st);
        env_update_left(bl, sr.mid, c->qn, c->W[j], *ch.Lenv[j], A.as<double>(), *left_env[k], eprec(c),
                        ch.err.as<unsigned>(), st);
        // serial chain continues left with A Lambda
        DBuf AL;
        AL.ensure(std::max<long long>(1, SA.size) * 8, st);
        scale_site(bl, sr.mid, c->qn, A.as<double>(), lamd.as<double>(), true, AL.as<double>(), st);
        ch.bond[b] = sr.mid;
        ch.lam[b] = sr.lam;
        env_alloc(*ch.Renv[b], sr.mid, c->W[j + 1].fl, eprec(c), st);
        env_update_right(sr.mid, br, c->qn, c->W[j + 1], *ch.Renv[j + 2], B.as<double>(), *ch.Renv[b], eprec(c),
                         ch.err.as<unsigned>(), st);
        ch.site[j] = std::move(AL);
        ch.site[j + 1] = std::move(B);
        ch.oc = j;
        std::vector<double> V(sr.lam.size());
        for (size_t i = 0; i < V.size(); ++i) V[i] = 1.0 / sr.lam[i];
        c->V[b] = V;
        c->Vbond[b] = sr.mid;
    }
    check_err_word(ch.err.as<unsigned>(), st);
    PD_CK(cudaStreamSynchronize(st));
    // hand the tensors to the regions
    c->bounds = bounds;
    c->reg.clear();
    for (int k = 0; k < R; ++k) {
        std::unique_ptr<Chain> r(new Chain());
        cudaStream_t rs;
        PD_CK(cudaStreamCreateWithFlags(&rs, cudaStreamNonBlocking));
        c->streams.s.push_back(rs);
        r->init(L, rs);
        r->own_stream = true;
        r->p = bounds[k];
        r->q = bounds[k + 1] - 1;
        for (int b = r->p; b <= r->q + 1; ++b) {
            r->bond[b] = ch.bond[b];
            r->lam[b] = ch.lam[b];
        }
        for (int sidx = r->p; sidx <= r->q; ++sidx) r->site[sidx] = std::move(ch.site[sidx]);
        if (k > 0) {
            r->site[r->p] = std::move(left_end[k]);
            r->Lenv[r->p] = std::move(left_env[k]);
        } else {
            r->Lenv[0] = std::move(ch.Lenv[0]);
        }
        for (int b = r->p + 1; b <= r->q + 1; ++b) r->Renv[b] = std::move(ch.Renv[b]);
        r->oc = r->p;
        r->rebind_all();
        c->reg.push_back(std::move(r));
    }
    // staggered start (Fig. 4): even regions (1-based) move to their right end
    std::vector<int> odd;
    for (int k = 1; k < R; k += 2) odd.push_back(k);
    if (p->serial_regions == 2) {
        lockstep_half(c, odd, std::vector<char>(odd.size(), 1), p);
        return;
    }
    parallel_items(odd, [&](int k) {
        region_half_sweep(c, *c->reg[k], true, p);
        check_err_word(c->reg[k]->err.as<unsigned>(), c->reg[k]->st);
    }, p->serial_regions != 0);
}

// One parallel sweep, Fig. 4 (a)-(d).
StepStats region_sweep(dmrg_ctx* c, const dmrg_sweep_params* p) {
    const int R = (int)c->reg.size();
    for (auto& r : c->reg) r->acc = StepStats();
    std::vector<int> all(R), mb, md;
    for (int k = 0; k < R; ++k) all[k] = k;
    for (int k = 1; k < R; k += 2) mb.push_back(k);
    for (int k = 2; k < R; k += 2) md.push_back(k);
    double e_last = 0.0;
    auto half = [&](bool first) {
        if (p->serial_regions == 2) {
            std::vector<char> dirs(R);
            for (int k = 0; k < R; ++k) dirs[k] = (k % 2 == 0) == first;
            lockstep_half(c, all, dirs, p);
            return;
        }
        parallel_items(all, [&](int k) {
            bool right = (k % 2 == 0) == first;
            region_half_sweep(c, *c->reg[k], right, p);
            check_err_word(c->reg[k]->err.as<unsigned>(), c->reg[k]->st);
        }, p->serial_regions != 0);
    };
    std::vector<double> e_merge(R, 0.0);
    half(true);                                                         // (a)
    parallel_items(mb, [&](int k) { do_merge(c, k, p, nullptr, &e_merge[k]); }, p->serial_regions != 0);   // (b)
    if (!mb.empty()) e_last = e_merge[mb.back()];
    half(false);                                                        // (c)
    parallel_items(md, [&](int k) { do_merge(c, k, p, nullptr, &e_merge[k]); }, p->serial_regions != 0);   // (d)
    if (!md.empty()) e_last = e_merge[md.back()];
    StepStats tot;
    for (auto& r : c->reg) tot.merge(r->acc);
    tot.energy = e_last;
    return tot;
}

}  // namespace

// ------------------------------------------------------------------------------------------
// C ABI
// ------------------------------------------------------------------------------------------
// The context's FP64-GEMM choice holds on the calling thread for the duration of the call.
struct EmuGuard {
    int saved, saved_qr;
    explicit EmuGuard(const dmrg_ctx* c) : saved(g_gemm64_emu), saved_qr(g_svd_qr) {
        g_gemm64_emu = (c && c->emu) ? 1 : 0;
        g_svd_qr = (c && c->svd_plain) ? 0 : 1;
    }
    ~EmuGuard() {
        g_gemm64_emu = saved;
        g_svd_qr = saved_qr;
    }
};
#define CTX_TRY try { EmuGuard emu_guard_(c);
#define CTX_CATCH(ctx)                                        \
    }                                                         \
    catch (const Error& e) {                                  \
        if (ctx) (ctx)->last_err = e.msg;                     \
        g_last_error = e.msg;                                 \
        return e.st;                                          \
    }                                                         \
    catch (const std::exception& e) {                         \
        if (ctx) (ctx)->last_err = e.what();                  \
        g_last_error = e.what();                              \
        return DMRG_ERR_STATE;                                \
    }

namespace {
// Work buffers come from the device's default stream-ordered pool.  With its default release
// threshold (0) every stream synchronisation hands freed memory back to the driver, and the next
// allocation maps it again; region threads that synchronise independently then spend their time
// re-mapping.  Keep freed memory in the pool instead (process-wide, set once).
void keep_pool_memory() {
    static const cudaError_t st = [] {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        cudaMemPool_t pool;
        e = cudaDeviceGetDefaultMemPool(&pool, dev);
        if (e != cudaSuccess) return e;
        uint64_t keep = UINT64_MAX;
        return cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }();
    PD_CK(st);
}
}  // namespace

extern "C" {

dmrg_status dmrg_init_mpo(dmrg_ctx** out, const dmrg_mpo_desc* mpo, const dmrg_config* cfg) {
    dmrg_ctx* c = nullptr;
    CTX_TRY
    PD_REQUIRE(out && mpo && cfg, DMRG_ERR_ARG, "null argument");
    *out = nullptr;
    PD_REQUIRE(mpo->n_sites >= 2 && mpo->d >= 1 && mpo->d <= 8, DMRG_ERR_ARG, "bad n_sites or d");
    PD_REQUIRE(mpo->qn_local && mpo->D && mpo->flux && mpo->W, DMRG_ERR_ARG, "null MPO array");
    PD_REQUIRE(cfg->precision == DMRG_FP64 || cfg->precision == DMRG_TF32 || cfg->precision == DMRG_BF16,
               DMRG_ERR_ARG, "unknown precision");
    PD_REQUIRE(cfg->precision == DMRG_FP64 || tc_available(), DMRG_ERR_STATE, "tensor-core engine unavailable");
    keep_pool_memory();
    std::unique_ptr<dmrg_ctx> C(new dmrg_ctx());
    c = C.get();
    C->L = mpo->n_sites;
    C->d = mpo->d;
    C->qtot = mpo->qn_total;
    C->qn.assign(mpo->qn_local, mpo->qn_local + mpo->d);
    C->prec = cfg->precision;
    C->kmax = cfg->kmax > 0 ? cfg->kmax : 8;
    C->svd_fp64 = cfg->svd_fp64 != 0;
    C->emu = cfg->fp64_emulation != 0;
    C->svd_plain = cfg->svd_plain_jacobi != 0;
    C->env64 = cfg->env_fp64 != 0;
    C->acc_edges = std::max(0, std::min(2, cfg->accurate_edges));
    PD_REQUIRE(!C->emu || tc_available(), DMRG_ERR_STATE, "FP64 emulation needs sm_103 tensor cores");
    PD_REQUIRE(C->kmax >= 2 && C->kmax <= 32, DMRG_ERR_ARG, "kmax must be in [2, 32]");
    C->base = (cudaStream_t)cfg->stream;
    PD_REQUIRE(mpo->D[0] == 1 && mpo->D[C->L] == 1, DMRG_ERR_ARG, "D[0] and D[L] must be 1");
    size_t woff = 0, foff = 0;
    for (int j = 0; j < C->L; ++j) {
        int Dl = mpo->D[j], Dr = mpo->D[j + 1];
        PD_REQUIRE(Dl > 0 && Dr > 0, DMRG_ERR_ARG, "MPO bond dimension must be positive");
        C->W.push_back(make_site_mpo(Dl, Dr, C->d, mpo->flux + foff, mpo->flux + foff + Dl, mpo->W + woff, C->qn));
        woff += (size_t)Dl * C->d * C->d * Dr;
        foff += Dl;
    }
    C->w12.resize(C->L);
    *out = C.release();
    return DMRG_OK;
    CTX_CATCH(c)
}

dmrg_status dmrg_set_mps(dmrg_ctx* c, const dmrg_mps_desc* m) {
    CTX_TRY
    PD_REQUIRE(c && m && m->n_sectors && m->sector_q && m->sector_m && m->data, DMRG_ERR_ARG, "null argument");
    c->ic.reset();
    c->reg.clear();
    c->bounds.clear();
    c->V.clear();
    c->Vbond.clear();
    c->serial.reset(new Chain());
    Chain& ch = *c->serial;
    ch.init(c->L, c->base);
    ch.p = 0;
    ch.q = c->L - 1;
    size_t so = 0;
    for (int b = 0; b <= c->L; ++b) {
        ch.bond[b] = make_sec(m->n_sectors[b], m->sector_q + so, m->sector_m + so);
        so += m->n_sectors[b];
    }
    PD_REQUIRE(ch.bond[0].n() == 1 && ch.bond[0].q[0] == 0 && ch.bond[0].m[0] == 1, DMRG_ERR_QN,
               "bond 0 must be the single sector {0: 1}");
    PD_REQUIRE(ch.bond[c->L].n() == 1 && ch.bond[c->L].q[0] == c->qtot && ch.bond[c->L].m[0] == 1, DMRG_ERR_QN,
               "bond L must be the single sector {qn_total: 1}");
    size_t off = 0;
    for (int j = 0; j < c->L; ++j) {
        const SiteLayout S = site_layout(ch.bond[j], ch.bond[j + 1], c->qn);
        ch.site[j].ensure(std::max<long long>(1, S.size) * 8, ch.st);
        if (S.size) PD_CK(cudaMemcpyAsync(ch.site[j].p, m->data + off, S.size * 8, cudaMemcpyHostToDevice, ch.st));
        off += S.size;
    }
    PD_CK(cudaStreamSynchronize(ch.st));
    int center = 0;
    if (m->canonical) {
        PD_REQUIRE(m->center >= 0 && m->center < c->L, DMRG_ERR_ARG, "centre outside the chain");
        center = m->center;
        ch.oc = center;
    } else {
        right_canonicalize(c, ch);
    }
    make_boundary_envs(c, ch);
    build_right_envs(c, ch, center + 1);
    for (int j = 0; j < center; ++j) {
        env_alloc(*ch.Lenv[j + 1], ch.bond[j + 1], c->W[j].fr, eprec(c), ch.st);
        env_update_left(ch.bond[j], ch.bond[j + 1], c->qn, c->W[j], *ch.Lenv[j], ch.site[j].as<double>(),
                        *ch.Lenv[j + 1], eprec(c), ch.err.as<unsigned>(), ch.st);
    }
    check_err_word(ch.err.as<unsigned>(), ch.st);
    c->dir = center < c->L - 1 ? 1 : -1;
    c->have_state = true;
    return DMRG_OK;
    CTX_CATCH(c)
}

dmrg_status dmrg_sweep(dmrg_ctx* c, const dmrg_sweep_params* p, dmrg_sweep_stats* stats) {
    CTX_TRY
    PD_REQUIRE(c && p, DMRG_ERR_ARG, "null argument");
    PD_REQUIRE(c->have_state, DMRG_ERR_STATE, "no state loaded");
    PD_REQUIRE(p->m_max >= 1 && p->dav_max_iter >= 1 && p->dav_tol >= 0, DMRG_ERR_ARG, "bad sweep parameters");
    c->ic.reset();
    auto t0 = std::chrono::steady_clock::now();
    StepStats tot;
    if (c->reg.empty()) {
        Chain& ch = *c->serial;
        ch.acc = StepStats();
        PD_REQUIRE(ch.oc == 0, DMRG_ERR_STATE, "serial sweep must start with the centre on site 0");
        for (int j = 0; j <= c->L - 2; ++j) bond_step(c, ch, j, true, p);
        for (int j = c->L - 2; j >= 0; --j) bond_step(c, ch, j, false, p);
        check_err_word(ch.err.as<unsigned>(), ch.st);
        tot = ch.acc;
        tot.energy = ch.acc.energy;
    } else {
        tot = region_sweep(c, p);
    }
    auto t1 = std::chrono::steady_clock::now();
    if (stats) {
        stats->energy = tot.energy;
        stats->max_trunc_err = tot.trunc;
        stats->max_m = tot.m;
        stats->n_matvec = tot.matvecs;
        stats->n_steps = tot.steps;
        stats->dav_nonconv = tot.nonconv;
        stats->seconds = std::chrono::duration<double>(t1 - t0).count();
        stats->matvec_seconds = tot.mv_ms * 1e-3;
        stats->matvec_flops = tot.mv_flops;
        stats->min_fidelity = tot.fid_min;
        stats->max_fidelity = tot.fid_max;
        stats->n_refine_matvec = tot.acc_matvecs;
        stats->refine_seconds = tot.acc_ms * 1e-3;
    }
    return DMRG_OK;
    CTX_CATCH(c)
}

dmrg_status dmrg_advance(dmrg_ctx* c, int n_steps, const dmrg_sweep_params* p, dmrg_sweep_stats* stats) {
    CTX_TRY
    PD_REQUIRE(c && p && n_steps >= 0, DMRG_ERR_ARG, "bad argument");
    PD_REQUIRE(c->have_state && c->reg.empty(), DMRG_ERR_STATE, "advance needs a serial state");
    PD_REQUIRE(p->m_max >= 1 && p->dav_max_iter >= 1 && p->dav_tol >= 0, DMRG_ERR_ARG, "bad sweep parameters");
    c->ic.reset();
    auto t0 = std::chrono::steady_clock::now();
    Chain& ch = *c->serial;
    ch.acc = StepStats();
    for (int i = 0; i < n_steps; ++i) {
        if (c->dir > 0 && ch.oc >= c->L - 1) c->dir = -1;
        if (c->dir < 0 && ch.oc <= 0) c->dir = 1;
        if (c->dir > 0) bond_step(c, ch, ch.oc, true, p);
        else bond_step(c, ch, ch.oc - 1, false, p);
    }
    check_err_word(ch.err.as<unsigned>(), ch.st);
    auto t1 = std::chrono::steady_clock::now();
    if (stats) {
        const StepStats& tot = ch.acc;
        stats->energy = tot.energy;
        stats->max_trunc_err = tot.trunc;
        stats->max_m = tot.m;
        stats->n_matvec = tot.matvecs;
        stats->n_steps = tot.steps;
        stats->dav_nonconv = tot.nonconv;
        stats->seconds = std::chrono::duration<double>(t1 - t0).count();
        stats->matvec_seconds = tot.mv_ms * 1e-3;
        stats->matvec_flops = tot.mv_flops;
        stats->min_fidelity = -1.0;
        stats->max_fidelity = -1.0;
        stats->n_refine_matvec = tot.acc_matvecs;
        stats->refine_seconds = tot.acc_ms * 1e-3;
    }
    return DMRG_OK;
    CTX_CATCH(c)
}

dmrg_status dmrg_setup_regions(dmrg_ctx* c, int n_regions, int warmup, const dmrg_sweep_params* p) {
    CTX_TRY
    PD_REQUIRE(c && p, DMRG_ERR_ARG, "null argument");
    PD_REQUIRE(c->have_state, DMRG_ERR_STATE, "no state loaded");
    PD_REQUIRE(n_regions >= 1 && warmup >= 0, DMRG_ERR_ARG, "bad region count or warm-up");
    PD_REQUIRE(c->reg.empty(), DMRG_ERR_STATE, "regions are already set up");
    c->ic.reset();
    if (n_regions == 1) return DMRG_OK;
    setup_regions(c, n_regions, warmup, p);
    return DMRG_OK;
    CTX_CATCH(c)
}

dmrg_status dmrg_merge(dmrg_ctx* c, int k, const dmrg_sweep_params* p, double* fidelity_out, double* energy_out) {
    CTX_TRY
    PD_REQUIRE(c && p, DMRG_ERR_ARG, "null argument");
    PD_REQUIRE(!c->reg.empty() && k >= 1 && k < (int)c->reg.size(), DMRG_ERR_ARG, "no such boundary");
    c->ic.reset();
    do_merge(c, k, p, fidelity_out, energy_out);
    return DMRG_OK;
    CTX_CATCH(c)
}

dmrg_status dmrg_energy(dmrg_ctx* c, double* E) {
    CTX_TRY
    PD_REQUIRE(c && E, DMRG_ERR_ARG, "null argument");
    PD_REQUIRE(c->have_state && c->reg.empty(), DMRG_ERR_STATE, "energy needs a serial state");
    Chain& ch = *c->serial;
    int j = std::min(ch.oc, c->L - 2);
    DBuf psi;
    form_psi(c, ch, j, psi);
    *E = rayleigh_fp64(c, ch, j, psi.as<double>());
    return DMRG_OK;
    CTX_CATCH(c)
}

dmrg_status dmrg_get_bond(dmrg_ctx* c, int b, int* q, int* m, int cap, int* n) {
    CTX_TRY
    PD_REQUIRE(c && n && c->have_state && b >= 0 && b <= c->L, DMRG_ERR_ARG, "bad argument");
    const Chain* ch = c->serial.get();
    if (!c->reg.empty())
        for (const auto& r : c->reg)
            if (b >= r->p && b <= r->q + 1) { ch = r.get(); break; }
    const Sec& s = ch->bond[b];
    *n = s.n();
    PD_REQUIRE(s.n() <= cap && q && m, DMRG_ERR_CAPACITY, "capacity too small");
    for (int i = 0; i < s.n(); ++i) { q[i] = s.q[i]; m[i] = s.m[i]; }
    return DMRG_OK;
    CTX_CATCH(c)
}

dmrg_status dmrg_get_lambda(dmrg_ctx* c, int b, double* lam, int cap, int* n) {
    CTX_TRY
    PD_REQUIRE(c && n && c->have_state && b >= 0 && b <= c->L, DMRG_ERR_ARG, "bad argument");
    const Chain* ch = c->serial.get();
    if (!c->reg.empty())
        for (const auto& r : c->reg)
            if (b >= r->p && b <= r->q + 1) { ch = r.get(); break; }
    const auto& v = ch->lam[b];
    *n = (int)v.size();
    PD_REQUIRE((int)v.size() <= cap && lam, DMRG_ERR_CAPACITY, "capacity too small");
    for (size_t i = 0; i < v.size(); ++i) lam[i] = v[i];
    return DMRG_OK;
    CTX_CATCH(c)
}

dmrg_status dmrg_energy_gradient(dmrg_ctx* c, double* Wbar, double* E) {
    CTX_TRY
    PD_REQUIRE(c && Wbar && c->have_state, DMRG_ERR_ARG, "bad argument");
    PD_REQUIRE(c->reg.empty(), DMRG_ERR_STATE, "the energy gradient needs a serial state");
    PD_REQUIRE(c->prec == DMRG_FP64, DMRG_ERR_STATE, "the energy gradient runs in FP64 mode");
    Chain& ch = *c->serial;
    const int L = c->L;
    cudaStream_t st = ch.st;
    // move the centre to site 0 by untruncated SVDs
    while (ch.oc > 0) gauge_step(c, ch, ch.oc - 1, false);
    std::vector<size_t> off(L + 1, 0);
    for (int j = 0; j < L; ++j) off[j + 1] = off[j] + c->W[j].W.size();
    double e_acc = 0.0;
    for (int j = 0; j + 1 < L; ++j) {
        DBuf psi;
        form_psi(c, ch, j, psi);
        const long long n = psi_layout(ch.bond[j], ch.bond[j + 2], c->qn).size;
        const double nrm2 = dot_host(psi.as<double>(), psi.as<double>(), n, st);
        PD_REQUIRE(nrm2 > 0.0, DMRG_ERR_NUMERIC, "zero two-site wavefunction");
        scale_vec(psi.as<double>(), n, 1.0 / std::sqrt(nrm2), st);
        const EnvSlab& Le = *ch.Lenv[j];
        const EnvSlab& Re = *ch.Renv[j + 2];
        DBuf Lp, Rp, xb, Lb, Rb;
        Lp.ensure(std::max<long long>(1, Le.lay.packed_size) * 8, st);
        Rp.ensure(std::max<long long>(1, Re.lay.packed_size) * 8, st);
        Lb.ensure(std::max<long long>(1, Le.lay.packed_size) * 8, st);
        Rb.ensure(std::max<long long>(1, Re.lay.packed_size) * 8, st);
        xb.ensure(std::max<long long>(1, n) * 8, st);
        env_to_packed(Le, Lp.as<double>(), st);
        env_to_packed(Re, Rp.as<double>(), st);
        // Phi = <psi, H_eff psi>: with ybar = psi the MPO gradient of site j is dE/dW_j (the other
        // sites sit in the environments); the last bond also gives site L - 1
        heff_backward(ch.bond[j], ch.bond[j + 2], c->qn, c->W[j], c->W[j + 1], Lp.as<double>(), Rp.as<double>(),
                      psi.as<double>(), psi.as<double>(), xb.as<double>(), Lb.as<double>(), Rb.as<double>(),
                      Wbar + off[j], j + 2 == L ? Wbar + off[j + 1] : nullptr, st);
        // xbar = H_eff^T psi, so <psi, xbar> = <psi|H_eff|psi>
        e_acc = dot_host(psi.as<double>(), xb.as<double>(), n, st);
        if (j + 2 < L) gauge_step(c, ch, j, true);
    }
    // back to site 0
    while (ch.oc > 0) gauge_step(c, ch, ch.oc - 1, false);
    if (E) *E = e_acc;
    return DMRG_OK;
    CTX_CATCH(c)
}

dmrg_status dmrg_get_site(dmrg_ctx* c, int j, double* out, long long cap, long long* n) {
    CTX_TRY
    PD_REQUIRE(c && n && c->have_state && j >= 0 && j < c->L, DMRG_ERR_ARG, "bad argument");
    Chain* ch = c->serial.get();
    int k = 0;
    if (!c->reg.empty()) {
        for (k = 0; k < (int)c->reg.size(); ++k)
            if (j >= c->reg[k]->p && j <= c->reg[k]->q) break;
        PD_REQUIRE(k < (int)c->reg.size(), DMRG_ERR_STATE, "site outside every region");
        ch = c->reg[k].get();
    }
    const SiteLayout S = site_layout(ch->bond[j], ch->bond[j + 1], c->qn);
    *n = S.size;
    PD_REQUIRE(S.size <= cap && out, DMRG_ERR_CAPACITY, "capacity too small");
    cudaStream_t st = ch->st;
    if (S.size && k > 0 && j == ch->p) {
        // first site of a region right of a boundary b = j: V_b = Lambda_b^-1 absorbed into its
        // rows, so the exported sites contract to ... psi_3 V psi_4 ... (Eq. merge)
        DBuf Vd, tmp;
        upload(Vd, c->V.at(j), st);
        tmp.ensure(S.size * 8, st);
        scale_site(ch->bond[j], ch->bond[j + 1], c->qn, ch->site[j].as<double>(), Vd.as<double>(), false,
                   tmp.as<double>(), st);
        PD_CK(cudaMemcpyAsync(out, tmp.p, S.size * 8, cudaMemcpyDeviceToHost, st));
        PD_CK(cudaStreamSynchronize(st));
    } else {
        if (S.size) PD_CK(cudaMemcpyAsync(out, ch->site[j].p, S.size * 8, cudaMemcpyDeviceToHost, st));
        PD_CK(cudaStreamSynchronize(st));
    }
    return DMRG_OK;
    CTX_CATCH(c)
}

dmrg_status dmrg_inverse_canonical(dmrg_ctx* c) {
    CTX_TRY
    PD_REQUIRE(c && c->have_state, DMRG_ERR_ARG, "bad argument");
    PD_REQUIRE(c->reg.empty(), DMRG_ERR_STATE, "the inverse canonical gauge is built from a serial state");
    Chain& ch = *c->serial;
    std::vector<const double*> sites(c->L);
    for (int j = 0; j < c->L; ++j) sites[j] = ch.site[j].as<double>();
    c->ic.reset();
    c->ic.reset(icmps_build(ch.bond, sites, ch.oc, c->qn, ch.st));
    return DMRG_OK;
    CTX_CATCH(c)
}

dmrg_status dmrg_icmps_bond(dmrg_ctx* c, int b, int* q, int* m, int cap, int* n) {
    CTX_TRY
    PD_REQUIRE(c && n && b >= 0 && b <= c->L, DMRG_ERR_ARG, "bad argument");
    PD_REQUIRE(c->ic != nullptr, DMRG_ERR_STATE, "no inverse canonical gauge built");
    const Sec& s = icmps_bond(*c->ic, b);
    *n = s.n();
    PD_REQUIRE(s.n() <= cap && q && m, DMRG_ERR_CAPACITY, "capacity too small");
    for (int i = 0; i < s.n(); ++i) { q[i] = s.q[i]; m[i] = s.m[i]; }
    return DMRG_OK;
    CTX_CATCH(c)
}

dmrg_status dmrg_icmps_v(dmrg_ctx* c, int b, double* v, int cap, int* n) {
    CTX_TRY
    PD_REQUIRE(c && n && b >= 0 && b <= c->L, DMRG_ERR_ARG, "bad argument");
    PD_REQUIRE(c->ic != nullptr, DMRG_ERR_STATE, "no inverse canonical gauge built");
    const auto& lam = icmps_lambda(*c->ic, b);
    *n = (int)lam.size();
    PD_REQUIRE((int)lam.size() <= cap && v, DMRG_ERR_CAPACITY, "capacity too small");
    for (size_t i = 0; i < lam.size(); ++i) v[i] = 1.0 / lam[i];
    return DMRG_OK;
    CTX_CATCH(c)
}

dmrg_status dmrg_icmps_site(dmrg_ctx* c, int j, double* out, long long cap, long long* n) {
    CTX_TRY
    PD_REQUIRE(c && n && j >= 0 && j < c->L, DMRG_ERR_ARG, "bad argument");
    PD_REQUIRE(c->ic != nullptr, DMRG_ERR_STATE, "no inverse canonical gauge built");
    const long long sz = icmps_site_size(*c->ic, j);
    *n = sz;
    PD_REQUIRE(sz <= cap && out, DMRG_ERR_CAPACITY, "capacity too small");
    cudaStream_t st = c->serial->st;
    if (sz) PD_CK(cudaMemcpyAsync(out, icmps_site_dev(*c->ic, j), sz * 8, cudaMemcpyDeviceToHost, st));
    PD_CK(cudaStreamSynchronize(st));
    return DMRG_OK;
    CTX_CATCH(c)
}

dmrg_status dmrg_local_expectations(dmrg_ctx* c, int n_ops1, const double* ops1, double* out1, int n_ops2,
                                    const double* ops2, double* out2, float* ms_out) {
    CTX_TRY
    PD_REQUIRE(c && n_ops1 >= 0 && n_ops2 >= 0, DMRG_ERR_ARG, "bad argument");
    PD_REQUIRE((n_ops1 == 0 || (ops1 && out1)) && (n_ops2 == 0 || (ops2 && out2)), DMRG_ERR_ARG, "null operator or output");
    PD_REQUIRE(c->ic != nullptr, DMRG_ERR_STATE, "no inverse canonical gauge built");
    icmps_expectations(*c->ic, c->qn, n_ops1, ops1, out1, n_ops2, ops2, out2, ms_out, c->serial->st);
    return DMRG_OK;
    CTX_CATCH(c)
}

dmrg_status dmrg_get_center(dmrg_ctx* c, int region, int* site) {
    CTX_TRY
    PD_REQUIRE(c && site && c->have_state, DMRG_ERR_ARG, "bad argument");
    if (c->reg.empty()) *site = c->serial->oc;
    else {
        PD_REQUIRE(region >= 0 && region < (int)c->reg.size(), DMRG_ERR_ARG, "no such region");
        *site = c->reg[region]->oc;
    }
    return DMRG_OK;
    CTX_CATCH(c)
}

dmrg_status dmrg_destroy(dmrg_ctx* c) {
    if (!c) return DMRG_OK;
    cudaStreamSynchronize(c->base);
    for (auto& r : c->reg)
        if (r->st) cudaStreamSynchronize(r->st);
    delete c;   // buffers free on their streams, then the owned streams are destroyed
    return DMRG_OK;
}

const char* dmrg_last_error(const dmrg_ctx* c) {
    if (c) return c->last_err.c_str();
    return g_last_error.c_str();
}

}  // extern "C"
