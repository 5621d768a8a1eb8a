// Inverse canonical MPS gauge and local expectation values (Sec. IV, Figs. 8 and 9).
//
// Gauge: psi_j = Lambda_j Gamma_j Lambda_{j+1} on every site and V_b = Lambda_b^-1 on every inner
// bond b (bond b joins sites b-1 and b), so that the state is psi_0 V_1 psi_1 ... V_{L-1} psi_{L-1}
// and every site tensor is an orthogonality centre (OC).  Built from a mixed-canonical state with
// its OC at site c in two untruncated passes of single-site SVDs:
//   (1) c, c-1, ..., 1: site j viewed as rows a x cols (s, b) = U Lambda W^T; site j <- W^T,
//       U Lambda absorbed into site j-1 (OC moves to site 0);
//   (2) 0, 1, ..., L-2: site j viewed as rows (a, s) x cols b = U Lambda W^T; psi_j <- U Lambda,
//       V_{j+1} <- Lambda^-1, Lambda W^T absorbed into site j+1.
// Pass (2) is Fig. 8's Lambda-V-Lambda step repeated at every bond: with site j+1 right-orthonormal,
// the SVD of the two-site Theta = psi_j B_{j+1} and that of psi_j share U and Lambda.  Singular
// values at or below 1e-12 of the largest are dropped so that V stays finite.
//
// Expectation values: every psi_j is an OC, so <O_j> needs only psi_j and a nearest-neighbour
// operator only Theta_j = psi_j V_{j+1} psi_{j+1}.  All sites and all bonds are measured at once:
//   colscale   P_j = psi_j V_{j+1}                         (one launch, every site)
//   GEMM       Theta_j = P_j psi_{j+1}                     (one grouped launch, every bond)
//   dots       Gram entries <X_p, X_p'> of equally charged blocks, chunked (one launch)
//   reduce     chunk partials -> Gram matrices in a fixed order (one launch)
//   contract   <O> = sum O[p,p'] G[p,p'] / tr G per operator and unit (one launch)
#include <map>

#include "plans.h"

namespace pd {
struct ICMPS;
}  // namespace pd

using namespace pd;

namespace {

const std::vector<int> kTrivial = {0};
constexpr int kDotChunk = 32768;     // elements per CTA in the chunked scale and dot launches

// out[off + e0 + e] = in[off + e0 + e] * v[voff + (e0 + e) % cols], e < len (one chunk of a block)
struct IcScale { long long off, voff; int e0, len, cols, pad_; };
__global__ void k_ic_colscale(const IcScale* __restrict__ jobs, const double* __restrict__ in,
                              const double* __restrict__ v, double* __restrict__ out) {
    const IcScale j = jobs[blockIdx.x];
    for (int e = threadIdx.x; e < j.len; e += blockDim.x) {
        const long long x = j.off + j.e0 + e;
        out[x] = in[x] * v[j.voff + (j.e0 + e) % j.cols];
    }
}

// part[t] = sum_e X[a + e] X[b + e], e < len; X = psi slab (slab 0) or Theta slab (slab 1)
struct IcDot { long long a, b; int len, slab; };
__global__ void k_ic_dot(const IcDot* __restrict__ jobs, const double* __restrict__ X0, const double* __restrict__ X1,
                         double* __restrict__ part) {
    const IcDot j = jobs[blockIdx.x];
    const double* X = j.slab ? X1 : X0;
    double s = 0.0;
    for (int e = threadIdx.x; e < j.len; e += blockDim.x) s = fma(X[j.a + e], X[j.b + e], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ double red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}

// G[gidx[e]] = sum of part[t0[e] .. t0[e+1]) in order
__global__ void k_ic_reduce(const int* __restrict__ t0, const int* __restrict__ gidx, const double* __restrict__ part,
                            int n, double* __restrict__ G) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int t = t0[e]; t < t0[e + 1]; ++t) s += part[t];
        G[gidx[e]] = s;
    }
}

// out[o * nu + u] = sum_{p,p'} O_o[p][p'] Gs[p][p'] / sum_p G[p][p], with Gs the symmetric
// completion of the upper triangle G[p][p'] (p <= p') of unit u (D x D at G + u * D * D).
__global__ void k_ic_contract(const double* __restrict__ G, const double* __restrict__ ops, int nops, int nu, int D,
                              double* __restrict__ out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nops * nu; i += gridDim.x * blockDim.x) {
        const int o = i / nu, u = i % nu;
        const double* g = G + (size_t)u * D * D;
        const double* op = ops + (size_t)o * D * D;
        double num = 0.0, den = 0.0;
        for (int p = 0; p < D; ++p) {
            den += g[p * D + p];
            for (int q = 0; q < D; ++q) num = fma(op[p * D + q], p <= q ? g[p * D + q] : g[q * D + p], num);
        }
        out[i] = den > 0.0 ? num / den : 0.0;
    }
}

inline unsigned gridn(long long n, int b) { return (unsigned)std::max<long long>(1, std::min<long long>((n + b - 1) / b, 65535)); }

// GEMM that absorbs a carry into a neighbouring site.
//   left = false: new[(t, s)] = carry[(i, 0)] site[(i, s)]  (carry blocks [mid_t][m_i], same charge)
//   left = true:  new[(x, s)] = site[(x, s)] carry[(i, 0)]  (carry blocks [m_i][mid_t], same charge)
void absorb(const Sec& carry_l, const Sec& carry_r, const Sec& site_l, const Sec& site_r, const std::vector<int>& qn,
            const double* carry, const double* site, bool carry_on_left, DBuf& out, Sec* new_l, Sec* new_r,
            cudaStream_t st) {
    GemmBatch g;
    const SiteLayout Sc = site_layout(carry_l, carry_r, kTrivial);
    if (!carry_on_left) {
        // carry: mid (rows) x site_l (cols); result bonds (carry_l = mid) x site_r
        const SiteLayout So = site_layout(site_l, site_r, qn);
        const SiteLayout Sn = site_layout(carry_l, site_r, qn);
        for (const auto& nb : Sn.blk) {
            const int io = site_l.find(carry_l.q[nb.i]);
            if (io < 0) continue;
            const int ob = So.at(io, nb.s), cb = Sc.at(nb.i, 0);
            if (ob < 0 || cb < 0) continue;
            // C(m = c, n = t) = sum_k site[k][c] carry[t][k]
            g.add(nb.cols, nb.rows, nb.off, 1, nb.cols, site_l.m[io], 1, 1, nb.cols,
                  {GSeg{So.blk[ob].off, Sc.blk[cb].off, site_l.m[io], 0}});
        }
        out.ensure(std::max<long long>(1, Sn.size) * 8, st);
        PD_CK(cudaMemsetAsync(out.p, 0, std::max<long long>(1, Sn.size) * 8, st));
        run_gemm64(g, site, carry, out.as<double>(), st);
        *new_l = carry_l;
        *new_r = site_r;
    } else {
        // carry: site_r (rows) x mid (cols); result bonds site_l x (carry_r = mid)
        const SiteLayout So = site_layout(site_l, site_r, qn);
        const SiteLayout Sn = site_layout(site_l, carry_r, qn);
        for (const auto& nb : Sn.blk) {
            const int io = site_r.find(carry_r.q[nb.j]);
            const int ob = So.at(nb.i, nb.s);
            if (io < 0 || ob < 0) continue;
            const int cb = Sc.at(carry_l.find(site_r.q[io]), 0);
            if (cb < 0) continue;
            // C(m = t, n = x) = sum_k carry[k][t] site[x][k]
            g.add(nb.cols, nb.rows, nb.off, 1, nb.cols, site_r.m[io], 1, 1, nb.cols,
                  {GSeg{Sc.blk[cb].off, So.blk[ob].off, site_r.m[io], 0}});
        }
        out.ensure(std::max<long long>(1, Sn.size) * 8, st);
        PD_CK(cudaMemsetAsync(out.p, 0, std::max<long long>(1, Sn.size) * 8, st));
        run_gemm64(g, carry, site, out.as<double>(), st);
        *new_l = site_l;
        *new_r = carry_r;
    }
}

}  // namespace

namespace pd {

// Host lists and device buffers of one measurement pass over a gauge (they depend only on its
// block structure and on which operator sets are measured), kept for later passes.
struct MeasPlan {
    bool with1 = false, with2 = false;
    std::vector<IcScale> scale;
    GemmBatch theta;
    std::vector<IcDot> dots;
    std::vector<int> t0, gidx;
    long long g_size = 0, g2_base = 0, p_size = 0, th_size = 0;
    DBuf dscale, ddots, dt0, dg, part, G, P, Th, o1, o2, dops1, dops2;
};

struct ICMPS {
    int L = 0;
    std::vector<Sec> bond;                    // L + 1
    std::vector<long long> site_off;          // L + 1, offsets into psi
    std::vector<long long> v_off;             // L + 1, offsets into V (bonds 1..L-1 used)
    std::vector<std::vector<double>> lam;     // L + 1 (host copies, sector order)
    DBuf psi, V;
    std::unique_ptr<MeasPlan> plan;           // last measurement plan
};


void icmps_free(ICMPS* p) { delete p; }

ICMPS* icmps_build(const std::vector<Sec>& bonds, const std::vector<const double*>& sites, int oc,
                   const std::vector<int>& qn, cudaStream_t st) {
    const int L = (int)sites.size();
    PD_REQUIRE(L >= 2 && (int)bonds.size() == L + 1 && oc >= 0 && oc < L, DMRG_ERR_ARG, "bad state for the gauge");
    std::unique_ptr<ICMPS> ic(new ICMPS());
    ic->L = L;
    std::vector<Sec> b = bonds;
    std::vector<DBuf> cur(L);
    for (int j = 0; j < L; ++j) {
        const long long n = site_layout(b[j], b[j + 1], qn).size;
        cur[j].ensure(std::max<long long>(1, n) * 8, st);
        if (n) PD_CK(cudaMemcpyAsync(cur[j].p, sites[j], n * 8, cudaMemcpyDeviceToDevice, st));
    }
    // (1) OC to site 0
    for (int j = oc; j >= 1; --j) {
        long long na, nb, nl;
        svd_split_bounds(b[j], b[j + 1], kTrivial, qn, &na, &nb, &nl);
        DBuf U, W;
        U.ensure(std::max<long long>(1, na) * 8, st);
        W.ensure(std::max<long long>(1, nb) * 8, st);
        SplitResult r = svd_split(b[j], b[j + 1], kTrivial, qn, cur[j].as<double>(), 1 << 30, 0.0, false, 1, 0,
                                  U.as<double>(), W.as<double>(), nullptr, st);
        DBuf nsite;
        Sec nl_, nr_;
        absorb(b[j], r.mid, b[j - 1], b[j], qn, U.as<double>(), cur[j - 1].as<double>(), true, nsite, &nl_, &nr_, st);
        PD_CK(cudaStreamSynchronize(st));
        cur[j] = std::move(W);
        cur[j - 1] = std::move(nsite);
        b[j] = r.mid;
    }
    // (2) Lambda V Lambda at every bond, left to right
    ic->lam.assign(L + 1, {});
    ic->lam[0] = {1.0};
    ic->lam[L] = {1.0};
    for (int j = 0; j + 1 < L; ++j) {
        long long na, nb, nl;
        svd_split_bounds(b[j], b[j + 1], qn, kTrivial, &na, &nb, &nl);
        DBuf A, W;
        A.ensure(std::max<long long>(1, na) * 8, st);
        W.ensure(std::max<long long>(1, nb) * 8, st);
        SplitResult r = svd_split(b[j], b[j + 1], qn, kTrivial, cur[j].as<double>(), 1 << 30, 1e-12, false, 1, 1,
                                  A.as<double>(), W.as<double>(), nullptr, st);
        DBuf nsite;
        Sec nl_, nr_;
        absorb(r.mid, b[j + 1], b[j + 1], b[j + 2], qn, W.as<double>(), cur[j + 1].as<double>(), false, nsite, &nl_,
               &nr_, st);
        PD_CK(cudaStreamSynchronize(st));
        cur[j] = std::move(A);
        cur[j + 1] = std::move(nsite);
        b[j + 1] = r.mid;
        ic->lam[j + 1] = r.lam;
    }
    // one slab for all site tensors, one for all V
    ic->bond = b;
    ic->site_off.assign(L + 1, 0);
    for (int j = 0; j < L; ++j) ic->site_off[j + 1] = ic->site_off[j] + site_layout(b[j], b[j + 1], qn).size;
    ic->psi.ensure(std::max<long long>(1, ic->site_off[L]) * 8, st);
    for (int j = 0; j < L; ++j) {
        const long long n = ic->site_off[j + 1] - ic->site_off[j];
        if (n) PD_CK(cudaMemcpyAsync(ic->psi.as<double>() + ic->site_off[j], cur[j].p, n * 8, cudaMemcpyDeviceToDevice, st));
    }
    ic->v_off.assign(L + 1, 0);
    std::vector<double> hv;
    for (int bb = 0; bb <= L; ++bb) {
        ic->v_off[bb] = (long long)hv.size();
        if (bb == 0 || bb == L) { hv.push_back(1.0); continue; }
        for (double x : ic->lam[bb]) hv.push_back(1.0 / x);
    }
    upload(ic->V, hv, st);
    PD_CK(cudaStreamSynchronize(st));
    return ic.release();
}

const Sec& icmps_bond(const ICMPS& ic, int b) { return ic.bond.at(b); }
const std::vector<double>& icmps_lambda(const ICMPS& ic, int b) { return ic.lam.at(b); }
long long icmps_site_size(const ICMPS& ic, int j) { return ic.site_off.at(j + 1) - ic.site_off.at(j); }
const double* icmps_site_dev(const ICMPS& ic, int j) { return ic.psi.as<double>() + ic.site_off.at(j); }

static std::unique_ptr<MeasPlan> make_meas_plan(const ICMPS& ic, const std::vector<int>& qn, bool with1, bool with2,
                                         cudaStream_t st) {
    const int L = ic.L, d = (int)qn.size(), D2 = d * d;
    std::unique_ptr<MeasPlan> M(new MeasPlan());
    M->with1 = with1;
    M->with2 = with2;
    std::vector<SiteLayout> S(L);
    for (int j = 0; j < L; ++j) S[j] = site_layout(ic.bond[j], ic.bond[j + 1], qn);
    struct Pair { long long a, b, len; };
    std::map<long long, std::vector<Pair>> gram;            // Gram element -> equally shaped block pairs
    M->g2_base = (long long)L * d * d;
    M->g_size = M->g2_base + (long long)std::max(0, L - 1) * D2 * D2;
    if (with1)
        for (int j = 0; j < L; ++j)
            for (int i = 0; i < ic.bond[j].n(); ++i)
                for (int s = 0; s < d; ++s)
                    for (int sp = s; sp < d; ++sp) {
                        if (qn[s] != qn[sp]) continue;
                        const int x = S[j].at(i, s), y = S[j].at(i, sp);
                        if (x < 0 || y < 0) continue;
                        const auto& bx = S[j].blk[x];
                        gram[((long long)j * d + s) * d + sp].push_back(
                            {ic.site_off[j] + bx.off, ic.site_off[j] + S[j].blk[y].off, (long long)bx.rows * bx.cols});
                    }
    // bonds: P_j = psi_j V_{j+1} (column scaling), Theta_j = P_j psi_{j+1}
    std::vector<long long> th_off(std::max(1, L), 0);
    if (with2) {
        for (int j = 0; j + 1 < L; ++j) {
            const Sec& bm = ic.bond[j + 1];
            std::vector<long long> moff(bm.n() + 1, 0);
            for (int t = 0; t < bm.n(); ++t) moff[t + 1] = moff[t] + bm.m[t];
            for (const auto& bk : S[j].blk) {
                const long long n = (long long)bk.rows * bk.cols;
                for (long long e0 = 0; e0 < n; e0 += kDotChunk)
                    M->scale.push_back({ic.site_off[j] + bk.off, ic.v_off[j + 1] + moff[bk.j], (int)e0,
                                        (int)std::min<long long>(kDotChunk, n - e0), bk.cols, 0});
            }
            const PsiLayout P = psi_layout(ic.bond[j], ic.bond[j + 2], qn);
            for (const auto& b : P.blk) {
                const int im = bm.find(ic.bond[j].q[b.i] + qn[b.s1]);
                if (im < 0) continue;
                const int lb = S[j].at(b.i, b.s1), rb = S[j + 1].at(im, b.s2);
                if (lb < 0 || rb < 0) continue;
                // C(m = c, n = a) = sum_mid psi_{j+1}[mid][c] P_j[a][mid]
                M->theta.add(b.cols, b.rows, th_off[j] + b.off, 1, b.cols, bm.m[im], 1, 1, b.cols,
                             {GSeg{ic.site_off[j + 1] + S[j + 1].blk[rb].off, ic.site_off[j] + S[j].blk[lb].off,
                                   bm.m[im], 0}});
            }
            for (int i = 0; i < ic.bond[j].n(); ++i)
                for (int p = 0; p < D2; ++p)
                    for (int pp = p; pp < D2; ++pp) {
                        const int s1 = p / d, s2 = p % d, t1 = pp / d, t2 = pp % d;
                        if (qn[s1] + qn[s2] != qn[t1] + qn[t2]) continue;
                        const int x = P.at(i, s1, s2), y = P.at(i, t1, t2);
                        if (x < 0 || y < 0) continue;
                        const auto& bx = P.blk[x];
                        gram[M->g2_base + ((long long)j * D2 + p) * D2 + pp].push_back(
                            {-1 - (th_off[j] + bx.off), th_off[j] + P.blk[y].off, (long long)bx.rows * bx.cols});
                    }
            th_off[j + 1] = th_off[j] + P.size;
        }
    }
    // flatten: one reduce entry per Gram element, its chunks contiguous in the listed order
    for (const auto& kv : gram) {
        M->t0.push_back((int)M->dots.size());
        M->gidx.push_back((int)kv.first);
        for (const auto& pr : kv.second) {
            const int slab = pr.a < 0 ? 1 : 0;
            const long long a = pr.a < 0 ? -1 - pr.a : pr.a;
            for (long long c = 0; c < pr.len; c += kDotChunk)
                M->dots.push_back({a + c, pr.b + c, (int)std::min<long long>(kDotChunk, pr.len - c), slab});
        }
    }
    M->t0.push_back((int)M->dots.size());
    PD_REQUIRE(M->dots.size() < (size_t)INT32_MAX && M->scale.size() < (size_t)INT32_MAX &&
                   M->g_size < (long long)INT32_MAX,
               DMRG_ERR_CAPACITY, "too many blocks to measure at once");
    upload(M->dscale, M->scale, st);
    upload(M->ddots, M->dots, st);
    upload(M->dt0, M->t0, st);
    upload(M->dg, M->gidx, st);
    M->part.ensure(std::max<size_t>(1, M->dots.size()) * 8, st);
    M->G.ensure(std::max<long long>(1, M->g_size) * 8, st);
    M->p_size = L > 1 ? ic.site_off[L - 1] : 0;
    M->th_size = L > 1 ? th_off[L - 1] : 0;
    if (with2) {
        M->P.ensure(std::max<long long>(1, M->p_size) * 8, st);
        M->Th.ensure(std::max<long long>(1, M->th_size) * 8, st);
        M->theta.upload_tiles(64, 64, st);
    }
    return M;
}

// ops1: [n1][d][d], ops2: [n2][d*d][d*d] (host); out1: [n1][L], out2: [n2][L-1] (host).
void icmps_expectations(ICMPS& ic, const std::vector<int>& qn, int n1, const double* ops1, double* out1, int n2,
                        const double* ops2, double* out2, float* ms_out, cudaStream_t st) {
    const int L = ic.L, d = (int)qn.size(), D2 = d * d;
    if (!ic.plan || ic.plan->with1 != (n1 > 0) || ic.plan->with2 != (n2 > 0))
        ic.plan = make_meas_plan(ic, qn, n1 > 0, n2 > 0, st);
    MeasPlan& M = *ic.plan;
    if (n1 > 0) upload(M.dops1, std::vector<double>(ops1, ops1 + (size_t)n1 * d * d), st);
    if (n2 > 0) upload(M.dops2, std::vector<double>(ops2, ops2 + (size_t)n2 * D2 * D2), st);
    M.o1.ensure(std::max(1, n1 * L) * 8, st);
    M.o2.ensure(std::max(1, n2 * std::max(1, L - 1)) * 8, st);
    PD_CK(cudaStreamSynchronize(st));
    // ---- device work ----
    cudaEvent_t e0, e1;
    PD_CK(cudaEventCreate(&e0));
    PD_CK(cudaEventCreate(&e1));
    PD_CK(cudaEventRecord(e0, st));
    PD_CK(cudaMemsetAsync(M.G.p, 0, std::max<long long>(1, M.g_size) * 8, st));
    if (n2 > 0 && !M.scale.empty()) {
        k_ic_colscale<<<(unsigned)M.scale.size(), 256, 0, st>>>(M.dscale.as<IcScale>(), ic.psi.as<double>(),
                                                               ic.V.as<double>(), M.P.as<double>());
        PD_LAUNCHED();
        PD_CK(cudaMemsetAsync(M.Th.p, 0, std::max<long long>(1, M.th_size) * 8, st));
        run_gemm64(M.theta, ic.psi.as<double>(), M.P.as<double>(), M.Th.as<double>(), st);
    }
    if (!M.dots.empty()) {
        k_ic_dot<<<(unsigned)M.dots.size(), 256, 0, st>>>(M.ddots.as<IcDot>(), ic.psi.as<double>(),
                                                          M.Th.as<double>(), M.part.as<double>());
        PD_LAUNCHED();
        const int ne = (int)M.gidx.size();
        k_ic_reduce<<<gridn(ne, 256), 256, 0, st>>>(M.dt0.as<int>(), M.dg.as<int>(), M.part.as<double>(), ne,
                                                    M.G.as<double>());
        PD_LAUNCHED();
    }
    if (n1 > 0) {
        k_ic_contract<<<gridn((long long)n1 * L, 128), 128, 0, st>>>(M.G.as<double>(), M.dops1.as<double>(), n1, L, d,
                                                                   M.o1.as<double>());
        PD_LAUNCHED();
    }
    if (n2 > 0 && L > 1) {
        k_ic_contract<<<gridn((long long)n2 * (L - 1), 128), 128, 0, st>>>(M.G.as<double>() + M.g2_base,
                                                                         M.dops2.as<double>(), n2, L - 1, D2,
                                                                         M.o2.as<double>());
        PD_LAUNCHED();
    }
    PD_CK(cudaEventRecord(e1, st));
    if (n1 > 0) PD_CK(cudaMemcpyAsync(out1, M.o1.p, (size_t)n1 * L * 8, cudaMemcpyDeviceToHost, st));
    if (n2 > 0 && L > 1) PD_CK(cudaMemcpyAsync(out2, M.o2.p, (size_t)n2 * (L - 1) * 8, cudaMemcpyDeviceToHost, st));
    PD_CK(cudaStreamSynchronize(st));
    float ms = 0.0f;
    PD_CK(cudaEventElapsedTime(&ms, e0, e1));
    PD_CK(cudaEventDestroy(e0));
    PD_CK(cudaEventDestroy(e1));
    if (ms_out) *ms_out = ms;
}

}  // namespace pd
