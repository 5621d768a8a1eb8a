// Contraction plans and device building blocks of the two-site DMRG step (Sec. II).
#include <cfloat>
#include <cmath>
#include <map>
#include <tuple>

#include "plans.h"

namespace pd {

thread_local int g_svd_qr = 1;

// ------------------------------------------------------------------------------------------
// Layouts
// ------------------------------------------------------------------------------------------
SiteLayout site_layout(const Sec& bl, const Sec& br, const std::vector<int>& qn) {
    SiteLayout L;
    L.d = (int)qn.size();
    L.index.assign((size_t)bl.n() * L.d, -1);
    long long off = 0;
    for (int i = 0; i < bl.n(); ++i)
        for (int s = 0; s < L.d; ++s) {
            int j = br.find(bl.q[i] + qn[s]);
            if (j < 0) continue;
            L.index[(size_t)i * L.d + s] = (int)L.blk.size();
            L.blk.push_back({i, s, j, off, bl.m[i], br.m[j]});
            off += (long long)bl.m[i] * br.m[j];
        }
    L.size = off;
    return L;
}

PsiLayout psi_layout2(const Sec& bl, const Sec& br, const std::vector<int>& qn1, const std::vector<int>& qn2) {
    PsiLayout P;
    P.d1 = (int)qn1.size();
    P.d2 = (int)qn2.size();
    P.d = P.d1;
    P.index.assign((size_t)bl.n() * P.d1 * P.d2, -1);
    long long off = 0;
    for (int i = 0; i < bl.n(); ++i)
        for (int s1 = 0; s1 < P.d1; ++s1)
            for (int s2 = 0; s2 < P.d2; ++s2) {
                int k = br.find(bl.q[i] + qn1[s1] + qn2[s2]);
                if (k < 0) continue;
                P.index[((size_t)i * P.d1 + s1) * P.d2 + s2] = (int)P.blk.size();
                P.blk.push_back({i, s1, s2, k, off, bl.m[i], br.m[k]});
                off += (long long)bl.m[i] * br.m[k];
            }
    P.size = off;
    return P;
}

PsiLayout psi_layout(const Sec& bl, const Sec& br, const std::vector<int>& qn) { return psi_layout2(bl, br, qn, qn); }

EnvLayout env_layout(const Sec& b, const std::vector<int>& flux, int ld) {
    EnvLayout E;
    E.D = (int)flux.size();
    E.ld = ld;
    E.index.assign((size_t)b.n() * E.D, -1);
    long long row = 0, packed = 0;
    for (int i = 0; i < b.n(); ++i)
        for (int w = 0; w < E.D; ++w) {
            int k = b.find(b.q[i] - flux[w]);
            if (k < 0) continue;
            E.index[(size_t)i * E.D + w] = (int)E.blk.size();
            E.blk.push_back({i, w, k, row, packed, b.m[i], b.m[k]});
            row += b.m[i];
            packed += (long long)b.m[i] * b.m[k];
        }
    E.rows = row;
    E.packed_size = packed;
    return E;
}

TwoSiteMPO two_site_mpo(const SiteMPO& a, const SiteMPO& b) {
    TwoSiteMPO T;
    const int d = a.d;
    T.D0 = a.Dl;
    T.D2 = b.Dr;
    T.d = d;
    T.f0 = a.fl;
    T.f2 = b.fr;
    std::vector<double> acc((size_t)a.Dl * d * d * d * d * b.Dr, 0.0);
    auto idx = [&](int w, int s1, int s1p, int s2, int s2p, int w2) {
        return (((((size_t)w * d + s1) * d + s1p) * d + s2) * d + s2p) * b.Dr + w2;
    };
    for (int w = 0; w < a.Dl; ++w)
        for (int s1 = 0; s1 < d; ++s1)
            for (int s1p = 0; s1p < d; ++s1p)
                for (int w1 = 0; w1 < a.Dr; ++w1) {
                    double x = a.at(w, s1, s1p, w1);
                    if (x == 0.0) continue;
                    for (int s2 = 0; s2 < d; ++s2)
                        for (int s2p = 0; s2p < d; ++s2p)
                            for (int w2 = 0; w2 < b.Dr; ++w2) {
                                double y = b.at(w1, s2, s2p, w2);
                                if (y != 0.0) acc[idx(w, s1, s1p, s2, s2p, w2)] += x * y;
                            }
                }
    for (int w = 0; w < a.Dl; ++w)
        for (int s1 = 0; s1 < d; ++s1)
            for (int s1p = 0; s1p < d; ++s1p)
                for (int s2 = 0; s2 < d; ++s2)
                    for (int s2p = 0; s2p < d; ++s2p)
                        for (int w2 = 0; w2 < b.Dr; ++w2) {
                            double v = acc[idx(w, s1, s1p, s2, s2p, w2)];
                            if (v != 0.0) T.nz.push_back({w, s1, s1p, s2, s2p, w2, v});
                        }
    return T;
}

// ------------------------------------------------------------------------------------------
// Batches and job lists
// ------------------------------------------------------------------------------------------
void GemmBatch::upload_tiles(int tm, int tn, cudaStream_t st) {
    if (tile_m == tm && tile_n == tn && dtiles.p) return;
    std::vector<GTile> tiles;
    for (int p = 0; p < (int)probs.size(); ++p)
        for (int m0 = 0; m0 < probs[p].M; m0 += tm)
            for (int n0 = 0; n0 < probs[p].N; n0 += tn) tiles.push_back({p, m0, n0, 0});
    ntiles = (int)tiles.size();
    upload(dprobs, probs, st);
    upload(dsegs, segs, st);
    upload(dtiles, tiles, st);
    tile_m = tm;
    tile_n = tn;
}

void run_gemm64(GemmBatch& g, const double* A, const double* B, double* C, cudaStream_t st) {
    if (g.empty()) return;
    if (g_gemm64_emu && run_gemm64_emu(g, A, B, C, st)) return;
    g.upload_tiles(64, 64, st);
    void* tok = prof_on() ? prof_start(st) : nullptr;
    launch_gemm_simt<double>(g.dprobs.as<GProb>(), g.dsegs.as<GSeg>(), g.dtiles.as<GTile>(), g.ntiles, A, B, C, st);
    if (tok) prof_stop(tok, st, g_prof_class == PROF_ENV ? PROF_ENV : PROF_F64, g.flops);
}

void run_gemm32(GemmBatch& g, const float* A, const float* B, float* C, cudaStream_t st) {
    if (g.empty()) return;
    g.upload_tiles(64, 64, st);
    void* tok = prof_on() ? prof_start(st) : nullptr;
    launch_gemm_simt<float>(g.dprobs.as<GProb>(), g.dsegs.as<GSeg>(), g.dtiles.as<GTile>(), g.ntiles, A, B, C, st);
    if (tok) prof_stop(tok, st, PROF_F32, g.flops);
}

template <class Tin>
void run_copy(const CopyList& c, const Tin* src, void* dst, Num out, cudaStream_t st) {
    if (c.jobs.empty()) return;
    const CopyJob* j = c.d.as<CopyJob>();
    const int2* ch = c.dc.as<int2>();
    int n = c.nchunks;
    if (out == Num::F64) launch_copy<Tin, double>(j, ch, n, src, (double*)dst, st);
    else if (out == Num::F32) launch_copy<Tin, float>(j, ch, n, src, (float*)dst, st);
    else launch_copy<Tin, __nv_bfloat16>(j, ch, n, src, (__nv_bfloat16*)dst, st);
}
template void run_copy<double>(const CopyList&, const double*, void*, Num, cudaStream_t);
template void run_copy<float>(const CopyList&, const float*, void*, Num, cudaStream_t);

template <>
void run_mix<double>(const MixList& m, const double* in, void* out, Num t, cudaStream_t st) {
    if (m.jobs.empty()) return;
    PD_REQUIRE(t == Num::F64, DMRG_ERR_ARG, "FP64 mix output must be FP64");
    launch_mix<double, double>(m.dj.as<MixJob>(), m.dc.as<int2>(), m.nchunks, m.dt.as<MixTerm>(), in, (double*)out, st);
}
template <>
void run_mix<float>(const MixList& m, const float* in, void* out, Num t, cudaStream_t st) {
    if (m.jobs.empty()) return;
    if (t == Num::F32)
        launch_mix<float, float>(m.dj.as<MixJob>(), m.dc.as<int2>(), m.nchunks, m.dt.as<MixTerm>(), in, (float*)out, st);
    else
        launch_mix<float, __nv_bfloat16>(m.dj.as<MixJob>(), m.dc.as<int2>(), m.nchunks, m.dt.as<MixTerm>(), in, (__nv_bfloat16*)out, st);
}

// ------------------------------------------------------------------------------------------
// Small helper kernels local to this file
// ------------------------------------------------------------------------------------------
namespace {

__global__ void k_scale_plain(double* x, long long n, double s) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        x[i] *= s;
}

// out block (rows x cols, row-major) = in block with column c scaled by v[voff + c].
struct ColScaleJob { long long src, dst, voff; int rows, cols; };
__global__ void k_colscale(const ColScaleJob* jobs, const double* in, const double* v, double* out) {
    const ColScaleJob j = jobs[blockIdx.y];
    long long total = (long long)j.rows * j.cols;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        int c = (int)(e % j.cols);
        out[j.dst + e] = in[j.src + e] * v[j.voff + c];
    }
}

// SVD scatter: write kept singular vectors into packed site-tensor blocks.
struct ScatJob {
    long long dst;       // output block offset
    long long base;      // W or V sector base offset
    long long s_off;     // sector offset into sig/order
    int rows, cols;      // output block shape
    int ld;              // column length of the source matrix (W: p, V: n)
    int off0;            // row offset inside the source column (r0 or c0)
    int fromW;           // 1: source columns in W (divide by sigma), 0: in V
    int left;            // 1: output [a][t] (t = kept index = column), 0: output [t][c]
    int lam_pow;         // multiply by lambda_t (normalised) when 1
    int pad_;
};
template <class T>
__global__ void k_svd_scatter(const ScatJob* jobs, const T* W, const T* V, const double* sig,
                              const int* order, const double* weights, double* out) {
    const ScatJob j = jobs[blockIdx.y];
    const double nrm = sqrt(weights[1]);
    long long total = (long long)j.rows * j.cols;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        int r = (int)(e / j.cols), c = (int)(e % j.cols);
        int t = j.left ? c : r;          // kept index
        int x = j.left ? r : c;          // position inside the source column
        int col = order[j.s_off + t];
        double sg = sig[j.s_off + col];
        double val = j.fromW ? (double)W[j.base + (long long)col * j.ld + j.off0 + x] / sg
                             : (double)V[j.base + (long long)col * j.ld + j.off0 + x];
        if (j.lam_pow) val *= sg / nrm;
        out[j.dst + e] = val;
    }
}

// lam_out[o + t] = sig[s_off + order[s_off + t]] / nrm
struct LamJob { long long s_off, o; int k, pad_; };
__global__ void k_lam_out(const LamJob* jobs, int njobs, const double* sig, const int* order, const double* weights,
                          double* lam) {
    const double nrm = sqrt(weights[1]);
    for (int b = blockIdx.x; b < njobs; b += gridDim.x) {
        LamJob j = jobs[b];
        for (int t = threadIdx.x; t < j.k; t += blockDim.x) lam[j.o + t] = sig[j.s_off + order[j.s_off + t]] / nrm;
    }
}

__global__ void k_place(double* G, int ldg, int k, const double* col, const double* row) {
    // G[i*ldg + k] = col[i] (i <= k);  G[k*ldg + i] = row[i] (i < k)
    for (int i = threadIdx.x; i <= k; i += blockDim.x) {
        G[(long long)i * ldg + k] = col[i];
        if (i < k) G[(long long)k * ldg + i] = row[i];
    }
}

inline int gridn(long long n, int cap = 2048) {
    long long g = (n + 255) / 256;
    return (int)std::max<long long>(1, std::min<long long>(g, cap));
}

}  // namespace

namespace {
struct RCJob { long long off, voff; int rows, cols, by_col, pad_; };
__global__ void k_rcscale(const RCJob* jobs, const double* in, const double* v, double* out) {
    const RCJob j = jobs[blockIdx.y];
    long long total = (long long)j.rows * j.cols;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        int r = (int)(e / j.cols), c = (int)(e % j.cols);
        out[j.off + e] = in[j.off + e] * v[j.voff + (j.by_col ? c : r)];
    }
}
}  // namespace

void scale_site(const Sec& bl, const Sec& br, const std::vector<int>& qn, const double* in, const double* lam,
                bool right_index, double* out, cudaStream_t st) {
    const SiteLayout S = site_layout(bl, br, qn);
    const Sec& vb = right_index ? br : bl;
    std::vector<long long> voff(vb.n() + 1, 0);
    for (int i = 0; i < vb.n(); ++i) voff[i + 1] = voff[i] + vb.m[i];
    std::vector<RCJob> jobs;
    int mx = 1;
    for (const auto& b : S.blk) {
        jobs.push_back({b.off, voff[right_index ? b.j : b.i], b.rows, b.cols, right_index ? 1 : 0, 0});
        mx = std::max(mx, b.rows * b.cols);
    }
    if (jobs.empty()) return;
    DBuf dj;
    upload(dj, jobs, st);
    k_rcscale<<<dim3(gridn(mx, 256), (unsigned)jobs.size()), 256, 0, st>>>(dj.as<RCJob>(), in, lam, out);
    PD_LAUNCHED();
    PD_CK(cudaStreamSynchronize(st));
}

namespace {
// T_j = 1.5 I - 0.5 G_j for square blocks (off, k)
struct NsJob { long long off; int k, pad_; };
__global__ void k_ns_prep(const NsJob* jobs, const double* G, double* T) {
    const NsJob j = jobs[blockIdx.y];
    long long total = (long long)j.k * j.k;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        int r = (int)(e / j.k), c = (int)(e % j.k);
        T[j.off + e] = (r == c ? 1.5 : 0.0) - 0.5 * G[j.off + e];
    }
}
}  // namespace

namespace {
// max over sectors of |G - I|_max, written by one block per sector into dev[s]
struct DevJob { long long off; int k, pad_; };
__global__ void k_gram_dev(const DevJob* jobs, const double* G, double* dev) {
    const DevJob j = jobs[blockIdx.x];
    double m = 0.0;
    const long long total = (long long)j.k * j.k;
    for (long long e = threadIdx.x; e < total; e += blockDim.x) {
        int r = (int)(e / j.k), c = (int)(e % j.k);
        m = fmax(m, fabs(G[j.off + e] - (r == c ? 1.0 : 0.0)));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ double red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) x = fmax(x, red[w]);
        dev[blockIdx.x] = x;
    }
}
}  // namespace

void orthonormalize_factor(const Sec& bl, const Sec& br, const std::vector<int>& qn, double* X, bool left,
                           cudaStream_t st) {
    const SiteLayout S = site_layout(bl, br, qn);
    const Sec& mid = left ? br : bl;            // the bond carrying the kept index
    std::vector<long long> goff(mid.n() + 1, 0);
    for (int i = 0; i < mid.n(); ++i) goff[i + 1] = goff[i] + (long long)mid.m[i] * mid.m[i];
    DBuf G, T, out, dev, dj, djd;
    G.ensure(std::max<long long>(1, goff.back()) * 8, st);
    T.ensure(std::max<long long>(1, goff.back()) * 8, st);
    out.ensure(std::max<long long>(1, S.size) * 8, st);
    dev.ensure(std::max(1, mid.n()) * 8, st);
    std::vector<NsJob> jobs;
    std::vector<DevJob> djobs;
    int mx = 1;
    for (int j = 0; j < mid.n(); ++j) {
        jobs.push_back({goff[j], mid.m[j], 0});
        djobs.push_back({goff[j], mid.m[j], 0});
        mx = std::max(mx, mid.m[j] * mid.m[j]);
    }
    upload(dj, jobs, st);
    upload(djd, djobs, st);
    GemmBatch gA;
    for (const auto& b : S.blk) {
        if (left) {
            int k = b.cols;   // A'[a][t] = sum_u A[a][u] T[u][t]:  C(m = t, n = a)
            gA.add(k, b.rows, b.off, 1, k, k, 1, 1, k, {GSeg{goff[b.j], b.off, k, 0}});
        } else {
            int k = b.rows;   // B'[t][c] = sum_u T[t][u] B[u][c]:  C(m = c, n = t)
            gA.add(b.cols, k, b.off, 1, b.cols, k, 1, 1, b.cols, {GSeg{b.off, goff[b.i], k, 0}});
        }
    }
    GemmBatch gG;
    std::vector<GemmBatch> per_block;
    if (left) {
        // G_j = sum over the blocks (a, s) of sector j of A^T A; all blocks share k_j columns
        std::vector<std::vector<GSeg>> segs(mid.n());
        for (const auto& b : S.blk) segs[b.j].push_back({b.off, b.off, b.rows, 0});
        for (int j = 0; j < mid.n(); ++j) gG.add(mid.m[j], mid.m[j], goff[j], 1, mid.m[j], 1, mid.m[j], 1, mid.m[j], segs[j]);
    } else {
        // G_j = sum over the blocks of B B^T; row strides differ per block, so one accumulating
        // launch per block (stream order serialises them)
        std::vector<int> first(mid.n(), 1);
        for (const auto& b : S.blk) {
            per_block.emplace_back();
            int k = b.rows;
            per_block.back().add(k, k, goff[b.i], b.cols, 1, b.cols, 1, 1, k, {GSeg{b.off, b.off, b.cols, 0}},
                                 first[b.i] ? 0 : 1);
            first[b.i] = 0;
        }
    }
    std::vector<double> hdev(mid.n());
    for (int iter = 0; iter < 6; ++iter) {
        PD_CK(cudaMemsetAsync(G.p, 0, std::max<long long>(1, goff.back()) * 8, st));
        if (left) run_gemm64(gG, X, X, G.as<double>(), st);
        else
            for (auto& g1 : per_block) run_gemm64(g1, X, X, G.as<double>(), st);
        k_gram_dev<<<mid.n(), 256, 0, st>>>(djd.as<DevJob>(), G.as<double>(), dev.as<double>());
        PD_LAUNCHED();
        PD_CK(cudaMemcpyAsync(hdev.data(), dev.p, mid.n() * 8, cudaMemcpyDeviceToHost, st));
        PD_CK(cudaStreamSynchronize(st));
        double worst = 0.0;
        for (double v : hdev) worst = std::max(worst, v);
        PD_REQUIRE(std::isfinite(worst) && worst < 0.9, DMRG_ERR_NUMERIC,
                   "kept singular vectors too far from orthonormal for the FP64 re-orthonormalisation (|I - X^T X| = " +
                       std::to_string(worst) + " at iteration " + std::to_string(iter) + ")");
        if (worst < 1e-13 || iter == 5) break;
        // X <- X (3I - G)/2 (left) or (3I - G)/2 X (right): one Newton-Schulz step
        k_ns_prep<<<dim3(gridn(mx, 256), (unsigned)jobs.size()), 256, 0, st>>>(dj.as<NsJob>(), G.as<double>(),
                                                                               T.as<double>());
        PD_LAUNCHED();
        if (left) run_gemm64(gA, T.as<double>(), X, out.as<double>(), st);
        else run_gemm64(gA, X, T.as<double>(), out.as<double>(), st);
        PD_CK(cudaMemcpyAsync(X, out.p, S.size * 8, cudaMemcpyDeviceToDevice, st));
    }
    PD_CK(cudaStreamSynchronize(st));
}

void convert_flat(const void* src, Num in, void* dst, Num out, long long n, cudaStream_t st) {
    if (n <= 0) return;
    CopyList cl;
    const long long chunk = 1 << 20;
    for (long long s0 = 0; s0 < n; s0 += chunk) {
        CopyJob j{};
        j.src = s0; j.dst = s0; j.rows = 1; j.cols = (int)std::min(chunk, n - s0);
        j.srs = 0; j.scs = 1; j.drs = 0; j.dcs = 1; j.zero_to = 0; j.scale = 1.0;
        cl.add(j);
    }
    cl.up(st);
    PD_REQUIRE(in == Num::F64 || in == Num::F32, DMRG_ERR_ARG, "convert_flat: source must be FP64 or FP32");
    if (in == Num::F64) run_copy<double>(cl, static_cast<const double*>(src), dst, out, st);
    else run_copy<float>(cl, static_cast<const float*>(src), dst, out, st);
}

void orthonormalize_square(const std::vector<SvdSec>& ss, double* V, cudaStream_t st) {
    std::vector<NsJob> jobs;
    std::vector<DevJob> djobs;
    GemmBatch gG, gX;
    long long tot = 0;
    int mx = 1;
    for (const auto& x : ss) {
        if (x.n <= 0) continue;
        const int n = x.n;
        jobs.push_back({x.v_off, n, 0});
        djobs.push_back({x.v_off, n, 0});
        mx = std::max(mx, n * n);
        // G = V^T V:  G(i, j) = sum_k V(k, i) V(k, j), V column-major (V(r, c) = V[off + r + c n])
        gG.add(n, n, x.v_off, n, 1, n, 1, n, 1, {GSeg{x.v_off, x.v_off, n, 0}});
        // V' = V T:   V'(r, c) = sum_u V(r, u) T(u, c), T symmetric
        gX.add(n, n, x.v_off, 1, n, n, 1, 1, n, {GSeg{x.v_off, x.v_off, n, 0}});
        tot = std::max(tot, x.v_off + (long long)n * n);
    }
    if (jobs.empty()) return;
    DBuf G, T, out, dev, dj, djd;
    G.ensure(tot * 8, st);
    T.ensure(tot * 8, st);
    out.ensure(tot * 8, st);
    dev.ensure(jobs.size() * 8, st);
    upload(dj, jobs, st);
    upload(djd, djobs, st);
    std::vector<double> hdev(jobs.size());
    for (int iter = 0; iter < 8; ++iter) {
        run_gemm64(gG, V, V, G.as<double>(), st);
        k_gram_dev<<<(unsigned)jobs.size(), 256, 0, st>>>(djd.as<DevJob>(), G.as<double>(), dev.as<double>());
        PD_LAUNCHED();
        PD_CK(cudaMemcpyAsync(hdev.data(), dev.p, jobs.size() * 8, cudaMemcpyDeviceToHost, st));
        PD_CK(cudaStreamSynchronize(st));
        double worst = 0.0;
        for (double v : hdev) worst = std::max(worst, v);
        PD_REQUIRE(std::isfinite(worst) && worst < 0.5, DMRG_ERR_NUMERIC,
                   "FP32 Jacobi rotations too far from orthogonal for the FP64 polish (|V^T V - I| = " +
                       std::to_string(worst) + " at iteration " + std::to_string(iter) + ")");
        if (worst < 1e-14) break;
        k_ns_prep<<<dim3(gridn(mx, 256), (unsigned)jobs.size()), 256, 0, st>>>(dj.as<NsJob>(), G.as<double>(),
                                                                               T.as<double>());
        PD_LAUNCHED();
        run_gemm64(gX, V, T.as<double>(), out.as<double>(), st);
        for (const auto& j : jobs)
            PD_CK(cudaMemcpyAsync(V + j.off, out.as<double>() + j.off, (size_t)j.k * j.k * 8, cudaMemcpyDeviceToDevice, st));
    }
}

void scale_vec(double* x, long long n, double s, cudaStream_t st) {
    if (n <= 0) return;
    k_scale_plain<<<gridn(n), 256, 0, st>>>(x, n, s);
    PD_LAUNCHED();
}

double dot_host(const double* x, const double* y, long long n, cudaStream_t st) {
    DBuf part, out;
    int nch = 64;
    part.ensure(sizeof(double) * nch, st);
    out.ensure(sizeof(double), st);
    launch_dots(x, 0, 1, y, n, part.as<double>(), nch, out.as<double>(), st);
    double h = 0.0;
    PD_CK(cudaMemcpyAsync(&h, out.p, sizeof(double), cudaMemcpyDeviceToHost, st));
    PD_CK(cudaStreamSynchronize(st));
    return h;
}

// ------------------------------------------------------------------------------------------
// Projected Hamiltonian plan: out = L x W1 x W2 x R applied to psi
// ------------------------------------------------------------------------------------------
std::unique_ptr<HeffPlan> make_heff_plan(const Sec& bl, const Sec& br, const std::vector<int>& qn,
                                         const TwoSiteMPO& w12, const EnvLayout& L, const EnvLayout& R,
                                         int prec, cudaStream_t st) {
    auto P = std::make_unique<HeffPlan>();
    const int d = (int)qn.size();
    P->prec = prec;
    P->psi = psi_layout(bl, br, qn);
    P->L = &L;
    P->R = &R;
    P->ld_psi = pad_ld(bl.maxm(), prec);
    P->ld_y = pad_ld(br.maxm(), prec);
    // FP64 plans read any stride (also the tensor-core layout of FP64-accurate mixed-mode
    // environments); the tensor-core plans need the 64-padded operand layout
    PD_REQUIRE(prec == DMRG_FP64 ? (L.ld >= bl.maxm() && R.ld >= br.maxm())
                                 : (L.ld == pad_ld(bl.maxm(), prec) && R.ld == pad_ld(br.maxm(), prec)),
               DMRG_ERR_STATE, "environment slab stride does not match the bond");
    const auto& pb = P->psi.blk;
    const int nb = (int)pb.size();

    // pack x (canonical [a][c]) into the transposed operand slab psiT ([c][a] rows)
    std::vector<long long> prow(nb);
    long long row = 0;
    for (int b = 0; b < nb; ++b) {
        prow[b] = row;
        CopyJob j{};
        j.src = pb[b].off; j.dst = row * P->ld_psi;
        j.rows = pb[b].cols; j.cols = pb[b].rows;
        j.srs = 1; j.scs = pb[b].cols; j.drs = P->ld_psi; j.dcs = 1;
        j.zero_to = kpad(pb[b].rows, prec); j.scale = 1.0;
        P->pack.add(j);
        row += pb[b].cols;
    }
    P->psiT_rows = row;

    // which (w, s1', s2') combinations feed anything
    std::vector<char> used((size_t)w12.D0 * d * d, 0);
    for (const auto& e : w12.nz) used[((size_t)e.w * d + e.s1p) * d + e.s2p] = 1;

    // L stage: X[w, b] = L_w psi_b, block [a_bra][c].  X blocks that feed exactly one Y block,
    // and that Y block has no other term, are written by the GEMM epilogue straight into the Y
    // operand slab (coefficient as alpha); only the rest goes through X and the mixing kernel.
    struct XB { int rows, cols, iab, lb, b; long long off; int fan; };
    std::vector<XB> xs;
    std::map<std::pair<int, int>, int> xidx;   // (w, b) -> X block
    for (int b = 0; b < nb; ++b) {
        const auto& B = pb[b];
        for (int w = 0; w < w12.D0; ++w) {
            if (!used[((size_t)w * d + B.s1) * d + B.s2]) continue;
            int iab = bl.find(bl.q[B.i] + w12.f0[w]);
            if (iab < 0) continue;
            int lb = L.at(iab, w);
            if (lb < 0) continue;
            xidx[{w, b}] = (int)xs.size();
            xs.push_back({bl.m[iab], B.cols, iab, lb, b, -1, 0});
        }
    }
    // MPO mix: Y[w2, o] = sum coef X[w, b]   (o = output block (iab, s1, s2))
    std::map<std::pair<int, int>, std::vector<std::pair<int, double>>> yterms;   // (o, w2)
    for (const auto& e : w12.nz) {
        for (int b = 0; b < nb; ++b) {
            const auto& B = pb[b];
            if (B.s1 != e.s1p || B.s2 != e.s2p) continue;
            auto it = xidx.find({e.w, b});
            if (it == xidx.end()) continue;
            int o = P->psi.at(xs[it->second].iab, e.s1, e.s2);
            if (o < 0) continue;
            int rb = R.at(pb[o].k, e.w2);
            if (rb < 0) continue;
            PD_REQUIRE(R.blk[rb].k == B.k, DMRG_ERR_QN, "MPO flux rule violated in the two-site operator");
            yterms[{o, e.w2}].push_back({it->second, e.v});
            xs[it->second].fan++;
        }
    }
    // Y slab rows
    long long yrow = 0;
    std::map<std::pair<int, int>, long long> yrow_of;
    for (auto& kv : yterms) {
        yrow_of[kv.first] = yrow;
        yrow += xs[kv.second.front().first].rows;
    }
    P->y_rows = yrow;
    // direct targets
    std::vector<long long> direct_row(xs.size(), -1);
    std::vector<double> direct_coef(xs.size(), 0.0);
    for (auto& kv : yterms)
        if (kv.second.size() == 1 && xs[kv.second[0].first].fan == 1) {
            direct_row[kv.second[0].first] = yrow_of[kv.first];
            direct_coef[kv.second[0].first] = kv.second[0].second;
        }
    long long xoff = 0;
    for (size_t xi = 0; xi < xs.size(); ++xi) {
        XB& x = xs[xi];
        const auto& B = pb[x.b];
        GSeg sg{prow[x.b] * P->ld_psi, L.blk[x.lb].row * L.ld, B.rows, 0};
        if (direct_row[xi] >= 0) {
            P->ldirect.add(x.cols, x.rows, direct_row[xi] * P->ld_y, P->ld_psi, 1, L.ld, 1, 1, P->ld_y, {sg}, 0,
                           direct_coef[xi]);
        } else {
            x.off = xoff;
            P->lstage.add(x.cols, x.rows, xoff, P->ld_psi, 1, L.ld, 1, 1, x.cols, {sg});
            xoff += (long long)x.rows * x.cols;
        }
    }
    P->x_size = xoff;
    // mixing jobs for the remaining Y blocks, R-stage segments for all of them
    std::map<int, std::vector<GSeg>> rsegs;
    for (auto& kv : yterms) {
        int o = kv.first.first, w2 = kv.first.second;
        const XB& x0 = xs[kv.second.front().first];
        const long long yr = yrow_of[kv.first];
        P->mix.flops += 2.0 * x0.rows * x0.cols * (double)kv.second.size();
        const bool direct = kv.second.size() == 1 && direct_row[kv.second[0].first] >= 0;
        if (!direct) {
            MixJob mj{};
            mj.dst = yr * P->ld_y;
            mj.rows = x0.rows;
            mj.cols = x0.cols;
            mj.ldo = P->ld_y;
            mj.zero_to = kpad(x0.cols, prec);
            mj.t0 = (int)P->mix.terms.size();
            mj.nt = (int)kv.second.size();
            for (auto& t : kv.second) P->mix.terms.push_back({xs[t.first].off, xs[t.first].cols, 0, t.second});
            P->mix.jobs.push_back(mj);
            P->mix.max_elems = std::max(P->mix.max_elems, mj.rows * std::max(mj.cols, mj.zero_to));
        }
        int rb = R.at(pb[o].k, w2);
        rsegs[o].push_back({R.blk[rb].row * R.ld, yr * P->ld_y, x0.cols, 0});
    }
    for (auto& kv : rsegs) {
        const auto& O = pb[kv.first];
        P->rstage.add(O.cols, O.rows, O.off, R.ld, 1, P->ld_y, 1, 1, O.cols, kv.second);
    }

    // diagonal
    for (int b = 0; b < nb; ++b) {
        const auto& B = pb[b];
        DiagJob j{};
        j.off = B.off; j.rows = B.rows; j.cols = B.cols; j.t0 = (int)P->dterms.size(); j.nt = 0;
        for (const auto& e : w12.nz) {
            if (e.s1 != B.s1 || e.s1p != B.s1 || e.s2 != B.s2 || e.s2p != B.s2) continue;
            if (w12.f0[e.w] != 0 || w12.f2[e.w2] != 0) continue;
            int lb = L.at(B.i, e.w), rb = R.at(B.k, e.w2);
            if (lb < 0 || rb < 0) continue;
            P->dterms.push_back({L.blk[lb].row * L.ld, R.blk[rb].row * R.ld, e.v});
            ++j.nt;
        }
        P->djobs.push_back(j);
        P->diag_max = std::max(P->diag_max, B.rows * B.cols);
    }

    P->flops = P->lstage.flops + P->ldirect.flops + P->rstage.flops + P->mix.flops;
    // upload static lists
    P->pack.up(st);
    P->mix.up(st);
    upload(P->ddj, P->djobs, st);
    upload(P->ddt, P->dterms, st);
    {
        std::vector<long long> el;
        for (const auto& j : P->djobs) el.push_back((long long)j.rows * j.cols);
        std::vector<int2> c = make_chunks(el);
        P->diag_chunks = (int)c.size();
        upload(P->ddc, c, st);
    }
    const Num t = mv_num(prec);
    P->psiT.ensure(std::max<long long>(1, P->psiT_rows) * P->ld_psi * num_size(t), st);
    P->Y.ensure(std::max<long long>(1, P->y_rows) * P->ld_y * num_size(t), st);
    // directly written Y blocks rely on zero padding columns: clear the slab once
    PD_CK(cudaMemsetAsync(P->Y.p, 0, std::max<long long>(1, P->y_rows) * P->ld_y * num_size(t), st));
    P->X.ensure(std::max<long long>(1, P->x_size) * (prec == DMRG_FP64 ? 8 : 4), st);
    PD_REQUIRE(P->psi.size < (1LL << 31), DMRG_ERR_CAPACITY, "two-site vector too long for one copy job");
    return P;
}

static const void* env_operand(const EnvSlab& e, int prec) {
    if (prec == DMRG_BF16) {
        PD_REQUIRE(e.op_valid, DMRG_ERR_STATE, "bf16 operand copy of an environment is stale");
        return e.op.p;
    }
    if ((prec == DMRG_TF32 || prec == PREC_F32) && e.num == Num::F64) {
        PD_REQUIRE(e.op32_valid, DMRG_ERR_STATE, "FP32 operand copy of an environment is stale");
        return e.op32.p;
    }
    return e.buf.p;
}

void heff_apply(HeffPlan& P, const EnvSlab& L, const EnvSlab& R, const double* x, double* y,
                unsigned* err, cudaStream_t st) {
    g_prof_class = PROF_MV;
    const int prec = P.prec;
    const Num t = mv_num(prec);
    run_copy<double>(P.pack, x, P.psiT.p, t, st);
    PD_CK(cudaMemsetAsync(y, 0, sizeof(double) * std::max<long long>(P.psi.size, 1), st));
    if (prec == DMRG_FP64) {
        run_gemm64(P.lstage, P.psiT.as<double>(), L.buf.as<double>(), P.X.as<double>(), st);
        run_gemm64(P.ldirect, P.psiT.as<double>(), L.buf.as<double>(), P.Y.as<double>(), st);
        run_mix<double>(P.mix, P.X.as<double>(), P.Y.p, Num::F64, st);
        run_gemm64(P.rstage, R.buf.as<double>(), P.Y.as<double>(), y, st);
    } else if (prec == PREC_F32) {
        // accurate refinement matvec: FP32 everywhere, FP64 output
        DBuf y32;
        y32.ensure(std::max<long long>(1, P.psi.size) * 4, st);
        PD_CK(cudaMemsetAsync(y32.p, 0, std::max<long long>(1, P.psi.size) * 4, st));
        const float* Lf = static_cast<const float*>(env_operand(L, PREC_F32));
        const float* Rf = static_cast<const float*>(env_operand(R, PREC_F32));
        run_gemm32(P.lstage, P.psiT.as<float>(), Lf, P.X.as<float>(), st);
        run_gemm32(P.ldirect, P.psiT.as<float>(), Lf, P.Y.as<float>(), st);
        run_mix<float>(P.mix, P.X.as<float>(), P.Y.p, Num::F32, st);
        run_gemm32(P.rstage, Rf, P.Y.as<float>(), y32.as<float>(), st);
        if (!P.unpack.d.p) {
            CopyJob j{};
            j.src = 0; j.dst = 0; j.rows = 1; j.cols = (int)P.psi.size; j.srs = 0; j.scs = 1; j.drs = 0; j.dcs = 1;
            j.zero_to = 0; j.scale = 1.0;
            P.unpack.add(j);
            P.unpack.up(st);
        }
        run_copy<float>(P.unpack, y32.as<float>(), y, Num::F64, st);
    } else {
        run_gemm_tc(P.lstage, t, P.psiT.p, P.psiT_rows, P.ld_psi, env_operand(L, prec), L.lay.rows, L.lay.ld,
                    P.X.p, Num::F32, err, st);
        run_gemm_tc(P.ldirect, t, P.psiT.p, P.psiT_rows, P.ld_psi, env_operand(L, prec), L.lay.rows, L.lay.ld,
                    P.Y.p, t, err, st);
        run_mix<float>(P.mix, P.X.as<float>(), P.Y.p, t, st);
        run_gemm_tc(P.rstage, t, env_operand(R, prec), R.lay.rows, R.lay.ld, P.Y.p, P.y_rows, P.ld_y, y, Num::F64,
                    err, st);
    }
}

void heff_diag(HeffPlan& P, const EnvSlab& L, const EnvSlab& R, double* out, cudaStream_t st) {
    if (P.djobs.empty()) return;
    if (L.num == Num::F64)
        launch_diag<double>(P.ddj.as<DiagJob>(), P.ddc.as<int2>(), P.diag_chunks, P.ddt.as<DiagTerm>(),
                            L.buf.as<double>(), L.lay.ld, R.buf.as<double>(), R.lay.ld, out, st);
    else
        launch_diag<float>(P.ddj.as<DiagJob>(), P.ddc.as<int2>(), P.diag_chunks, P.ddt.as<DiagTerm>(),
                           L.buf.as<float>(), L.lay.ld, R.buf.as<float>(), R.lay.ld, out, st);
}

// ------------------------------------------------------------------------------------------
// Environment slabs
// ------------------------------------------------------------------------------------------
void env_alloc(EnvSlab& e, const Sec& b, const std::vector<int>& flux, int prec, cudaStream_t st) {
    e.lay = env_layout(b, flux, pad_ld(b.maxm(), prec));
    e.num = env_num(prec);
    size_t bytes = (size_t)std::max<long long>(1, e.lay.rows) * e.lay.ld * num_size(e.num);
    e.buf.ensure(bytes, st);
    PD_CK(cudaMemsetAsync(e.buf.p, 0, bytes, st));
    e.op_valid = false;
    e.op32_valid = false;
    e.valid = true;
}

void env_make_operand(EnvSlab& e, int prec, cudaStream_t st) {
    const bool bf = prec == DMRG_BF16, f32 = (prec == DMRG_TF32 || prec == PREC_F32) && e.num == Num::F64;
    if ((!bf && !f32) || (bf && e.op_valid) || (f32 && e.op32_valid)) return;
    CopyList c;
    long long n = std::max<long long>(1, e.lay.rows) * e.lay.ld;
    // one flat row-major copy of the whole slab (padding included, zeros stay zeros)
    const long long chunk = 1 << 20;
    for (long long s = 0; s < n; s += chunk) {
        CopyJob j{};
        j.src = s; j.dst = s; j.rows = 1; j.cols = (int)std::min(chunk, n - s);
        j.srs = 0; j.scs = 1; j.drs = 0; j.dcs = 1; j.zero_to = 0; j.scale = 1.0;
        c.add(j);
    }
    c.up(st);
    DBuf& dst = bf ? e.op : e.op32;
    dst.ensure(n * (bf ? 2 : 4), st);
    if (e.num == Num::F64) run_copy<double>(c, e.buf.as<double>(), dst.p, bf ? Num::BF16 : Num::F32, st);
    else run_copy<float>(c, e.buf.as<float>(), dst.p, Num::BF16, st);
    (bf ? e.op_valid : e.op32_valid) = true;
}

void env_from_packed(EnvSlab& e, const double* packed, cudaStream_t st) {
    CopyList c;
    for (const auto& b : e.lay.blk) {
        CopyJob j{};
        j.src = b.packed; j.dst = b.row * e.lay.ld; j.rows = b.rows; j.cols = b.cols;
        j.srs = b.cols; j.scs = 1; j.drs = e.lay.ld; j.dcs = 1; j.zero_to = 0; j.scale = 1.0;
        c.add(j);
    }
    c.up(st);
    run_copy<double>(c, packed, e.buf.p, e.num, st);
    e.op_valid = false;
    e.op32_valid = false;
    e.valid = true;
}

void env_to_packed(const EnvSlab& e, double* packed, cudaStream_t st) {
    CopyList c;
    for (const auto& b : e.lay.blk) {
        CopyJob j{};
        j.src = b.row * e.lay.ld; j.dst = b.packed; j.rows = b.rows; j.cols = b.cols;
        j.srs = e.lay.ld; j.scs = 1; j.drs = b.cols; j.dcs = 1; j.zero_to = 0; j.scale = 1.0;
        c.add(j);
    }
    c.up(st);
    if (e.num == Num::F64) run_copy<double>(c, e.buf.as<double>(), packed, Num::F64, st);
    else run_copy<float>(c, e.buf.as<float>(), packed, Num::F64, st);
    PD_CK(cudaStreamSynchronize(st));   // the job list is freed on return
}

void env_boundary(EnvSlab& e, const Sec& b, const std::vector<int>& flux, int prec, cudaStream_t st) {
    env_alloc(e, b, flux, prec, st);
    PD_REQUIRE(e.lay.blk.size() == 1 && e.lay.blk[0].rows == 1 && e.lay.blk[0].cols == 1, DMRG_ERR_QN,
               "boundary environment is not a single 1x1 block");
    if (e.num == Num::F64) {
        double one = 1.0;
        PD_CK(cudaMemcpyAsync(e.buf.p, &one, 8, cudaMemcpyHostToDevice, st));
    } else {
        float one = 1.0f;
        PD_CK(cudaMemcpyAsync(e.buf.p, &one, 4, cudaMemcpyHostToDevice, st));
    }
    PD_CK(cudaStreamSynchronize(st));
    e.op_valid = false;
    e.op32_valid = false;
}

// ------------------------------------------------------------------------------------------
// Environment updates (Sec. II operator transformation)
// ------------------------------------------------------------------------------------------
// Environment updates compound their rounding errors site after site, so they run at FP32
// accuracy or better in every mode: FP64 GEMMs in FP64 mode and, with FP64-accurate environments,
// in the mixed modes (PREC_ENV64, on the tensor-core operand layout); FP32 SIMT GEMMs otherwise.
static void run_env_gemm(GemmBatch& g, int prec, const void* A, long long arows, int lda, const void* B,
                         long long brows, int ldb, void* C, unsigned* err, cudaStream_t st) {
    (void)arows; (void)lda; (void)brows; (void)ldb; (void)err;
    if (g.empty()) return;
    if (env_num(prec) == Num::F64) run_gemm64(g, (const double*)A, (const double*)B, (double*)C, st);
    else run_gemm32(g, (const float*)A, (const float*)B, (float*)C, st);
}

namespace {
// Environment-update GEMMs are tallied as such; the calling thread's class is restored on return.
struct EnvProfClass {
    int saved = g_prof_class;
    EnvProfClass() { g_prof_class = PROF_ENV; }
    ~EnvProfClass() { g_prof_class = saved; }
};
}  // namespace

void env_update_left(const Sec& ba, const Sec& bb, const std::vector<int>& qn, const SiteMPO& W,
                     const EnvSlab& Lin, const double* A, EnvSlab& Lout, int prec, unsigned* err, cudaStream_t st) {
    EnvProfClass prof_class;
    const int d = (int)qn.size();
    const SiteLayout S = site_layout(ba, bb, qn);
    const EnvLayout& Li = Lin.lay;
    const Num tn = env_num(prec);
    const int ldS = pad_ld(ba.maxm(), prec);
    // A^T slab: block (ia, s) rows b, cols a
    CopyList pk;
    std::vector<long long> srow(S.blk.size());
    long long row = 0;
    for (size_t b = 0; b < S.blk.size(); ++b) {
        const auto& B = S.blk[b];
        srow[b] = row;
        CopyJob j{};
        j.src = B.off; j.dst = row * ldS; j.rows = B.cols; j.cols = B.rows;
        j.srs = 1; j.scs = B.cols; j.drs = ldS; j.dcs = 1; j.zero_to = kpad(B.rows, prec); j.scale = 1.0;
        pk.add(j);
        row += B.cols;
    }
    const long long srows = row;
    // which (w, s') pairs feed anything
    std::vector<char> usedws((size_t)W.Dl * d, 0);
    for (int w = 0; w < W.Dl; ++w)
        for (int s = 0; s < d; ++s)
            for (int sp = 0; sp < d; ++sp)
                for (int wp = 0; wp < W.Dr; ++wp)
                    if (W.at(w, s, sp, wp) != 0.0) usedws[(size_t)w * d + sp] = 1;
    // stage 1: T1(iab, w, s') [b][a_bra] = L_w A_s'
    struct TB { long long off; int rows, cols; };   // rows = b, cols = a_bra
    std::map<std::tuple<int, int, int>, TB> t1;
    GemmBatch g1;
    long long toff = 0;
    for (const auto& lb : Li.blk) {
        for (int sp = 0; sp < d; ++sp) {
            if (!usedws[(size_t)lb.w * d + sp]) continue;
            int ab = S.at(lb.k, sp);
            if (ab < 0) continue;
            const auto& AB = S.blk[ab];
            TB t{toff, AB.cols, lb.rows};
            t1[{lb.i, lb.w, sp}] = t;
            g1.add(lb.rows, AB.cols, toff, Li.ld, 1, ldS, 1, 1, lb.rows,
                   {GSeg{lb.row * Li.ld, srow[ab] * ldS, lb.cols, 0}});
            toff += (long long)t.rows * t.cols;
        }
    }
    // stage 2: T2(w', s, iab) [b][a_bra] = sum W[w,s,s',w'] T1(iab, w, s')
    const EnvLayout& Lo = Lout.lay;
    const int ldT = pad_ld(ba.maxm(), prec);
    MixList mx;
    std::map<std::tuple<int, int, int>, long long> t2row;
    std::map<std::tuple<int, int, int>, std::vector<std::pair<const TB*, double>>> t2terms;
    for (const auto& kv : t1) {
        int iab, w, sp;
        std::tie(iab, w, sp) = kv.first;
        for (int s = 0; s < d; ++s)
            for (int wp = 0; wp < W.Dr; ++wp) {
                double c = W.at(w, s, sp, wp);
                if (c == 0.0) continue;
                if (S.at(iab, s) < 0) continue;
                int ibb = bb.find(ba.q[iab] + qn[s]);
                if (ibb < 0 || Lo.at(ibb, wp) < 0) continue;
                t2terms[{wp, s, iab}].push_back({&kv.second, c});
            }
    }
    long long trow = 0;
    for (auto& kv : t2terms) {
        const TB* x0 = kv.second.front().first;
        t2row[kv.first] = trow;
        MixJob mj{};
        mj.dst = trow * ldT; mj.rows = x0->rows; mj.cols = x0->cols; mj.ldo = ldT;
        mj.zero_to = kpad(x0->cols, prec); mj.t0 = (int)mx.terms.size(); mj.nt = (int)kv.second.size();
        for (auto& t : kv.second) mx.terms.push_back({t.first->off, t.first->cols, 0, t.second});
        mx.jobs.push_back(mj);
        mx.max_elems = std::max(mx.max_elems, mj.rows * std::max(mj.cols, mj.zero_to));
        trow += x0->rows;
    }
    // stage 3: Lout(ibb, w') [b_bra][b] = sum_{s, iab} A_s^T T2(w', s, iab)
    GemmBatch g3;
    for (const auto& ob : Lo.blk) {
        std::vector<GSeg> sg;
        for (int s = 0; s < d; ++s) {
            int iab = ba.find(bb.q[ob.i] - qn[s]);
            if (iab < 0) continue;
            int ab = S.at(iab, s);
            if (ab < 0) continue;
            auto it = t2row.find({ob.w, s, iab});
            if (it == t2row.end()) continue;
            sg.push_back({it->second * ldT, srow[ab] * ldS, ba.m[iab], 0});
        }
        g3.add(ob.cols, ob.rows, ob.row * Lo.ld, ldT, 1, ldS, 1, 1, Lo.ld, sg);
    }
    // execute
    pk.up(st);
    mx.up(st);
    DBuf sl, t1b, t2b;
    sl.ensure(std::max<long long>(1, srows) * ldS * num_size(tn), st);
    t1b.ensure(std::max<long long>(1, toff) * num_size(tn), st);
    t2b.ensure(std::max<long long>(1, trow) * ldT * num_size(tn), st);
    run_copy<double>(pk, A, sl.p, tn, st);
    run_env_gemm(g1, prec, Lin.buf.p, Li.rows, Li.ld, sl.p, srows, ldS, t1b.p, err, st);
    if (tn == Num::F64) run_mix<double>(mx, t1b.as<double>(), t2b.p, tn, st);
    else run_mix<float>(mx, t1b.as<float>(), t2b.p, tn, st);
    run_env_gemm(g3, prec, t2b.p, trow, ldT, sl.p, srows, ldS, Lout.buf.p, err, st);
    Lout.op_valid = false;
    Lout.op32_valid = false;
    PD_CK(cudaStreamSynchronize(st));   // scratch and job lists are released on return
}

void env_update_right(const Sec& ba, const Sec& bc, const std::vector<int>& qn, const SiteMPO& W,
                      const EnvSlab& Rin, const double* Bt, EnvSlab& Rout, int prec, unsigned* err, cudaStream_t st) {
    EnvProfClass prof_class;
    const int d = (int)qn.size();
    const SiteLayout S = site_layout(ba, bc, qn);
    const EnvLayout& Ri = Rin.lay;
    const Num tn = env_num(prec);
    const int ldS = pad_ld(bc.maxm(), prec);
    // B slab: block (ia, s) rows a, cols c (same orientation as the packed block)
    CopyList pk;
    std::vector<long long> srow(S.blk.size());
    long long row = 0;
    for (size_t b = 0; b < S.blk.size(); ++b) {
        const auto& B = S.blk[b];
        srow[b] = row;
        CopyJob j{};
        j.src = B.off; j.dst = row * ldS; j.rows = B.rows; j.cols = B.cols;
        j.srs = B.cols; j.scs = 1; j.drs = ldS; j.dcs = 1; j.zero_to = kpad(B.cols, prec); j.scale = 1.0;
        pk.add(j);
        row += B.rows;
    }
    const long long srows = row;
    std::vector<char> usedws((size_t)W.Dr * d, 0);   // (w', s')
    for (int w = 0; w < W.Dl; ++w)
        for (int s = 0; s < d; ++s)
            for (int sp = 0; sp < d; ++sp)
                for (int wp = 0; wp < W.Dr; ++wp)
                    if (W.at(w, s, sp, wp) != 0.0) usedws[(size_t)wp * d + sp] = 1;
    // stage 1: T1(icb, w', s') [a][c_bra] = R_w' B_s'^T
    struct TB { long long off; int rows, cols; };   // rows = a, cols = c_bra
    std::map<std::tuple<int, int, int>, TB> t1;
    GemmBatch g1;
    long long toff = 0;
    for (const auto& rb : Ri.blk) {
        for (int sp = 0; sp < d; ++sp) {
            if (!usedws[(size_t)rb.w * d + sp]) continue;
            int ia = ba.find(bc.q[rb.k] - qn[sp]);
            if (ia < 0) continue;
            int bbk = S.at(ia, sp);
            if (bbk < 0) continue;
            const auto& BB = S.blk[bbk];
            TB t{toff, BB.rows, rb.rows};
            t1[{rb.i, rb.w, sp}] = t;
            g1.add(rb.rows, BB.rows, toff, Ri.ld, 1, ldS, 1, 1, rb.rows,
                   {GSeg{rb.row * Ri.ld, srow[bbk] * ldS, rb.cols, 0}});
            toff += (long long)t.rows * t.cols;
        }
    }
    // stage 2: T2(w, s, icb) [a][c_bra] = sum W[w,s,s',w'] T1(icb, w', s')
    const EnvLayout& Ro = Rout.lay;
    const int ldT = pad_ld(bc.maxm(), prec);
    MixList mx;
    std::map<std::tuple<int, int, int>, long long> t2row;
    std::map<std::tuple<int, int, int>, std::vector<std::pair<const TB*, double>>> t2terms;
    for (const auto& kv : t1) {
        int icb, wp, sp;
        std::tie(icb, wp, sp) = kv.first;
        for (int w = 0; w < W.Dl; ++w)
            for (int s = 0; s < d; ++s) {
                double c = W.at(w, s, sp, wp);
                if (c == 0.0) continue;
                int iab = ba.find(bc.q[icb] - qn[s]);
                if (iab < 0 || S.at(iab, s) < 0) continue;
                if (Ro.at(iab, w) < 0) continue;
                t2terms[{w, s, icb}].push_back({&kv.second, c});
            }
    }
    long long trow = 0;
    for (auto& kv : t2terms) {
        const TB* x0 = kv.second.front().first;
        t2row[kv.first] = trow;
        MixJob mj{};
        mj.dst = trow * ldT; mj.rows = x0->rows; mj.cols = x0->cols; mj.ldo = ldT;
        mj.zero_to = kpad(x0->cols, prec); mj.t0 = (int)mx.terms.size(); mj.nt = (int)kv.second.size();
        for (auto& t : kv.second) mx.terms.push_back({t.first->off, t.first->cols, 0, t.second});
        mx.jobs.push_back(mj);
        mx.max_elems = std::max(mx.max_elems, mj.rows * std::max(mj.cols, mj.zero_to));
        trow += x0->rows;
    }
    // stage 3: Rout(iab, w) [a_bra][a] = sum_{s, icb} B_s T2(w, s, icb)^T
    GemmBatch g3;
    for (const auto& ob : Ro.blk) {
        std::vector<GSeg> sg;
        for (int s = 0; s < d; ++s) {
            int icb = bc.find(ba.q[ob.i] + qn[s]);
            if (icb < 0) continue;
            int bbk = S.at(ob.i, s);
            if (bbk < 0) continue;
            auto it = t2row.find({ob.w, s, icb});
            if (it == t2row.end()) continue;
            sg.push_back({it->second * ldT, srow[bbk] * ldS, bc.m[icb], 0});
        }
        g3.add(ob.cols, ob.rows, ob.row * Ro.ld, ldT, 1, ldS, 1, 1, Ro.ld, sg);
    }
    pk.up(st);
    mx.up(st);
    DBuf sl, t1b, t2b;
    sl.ensure(std::max<long long>(1, srows) * ldS * num_size(tn), st);
    t1b.ensure(std::max<long long>(1, toff) * num_size(tn), st);
    t2b.ensure(std::max<long long>(1, trow) * ldT * num_size(tn), st);
    run_copy<double>(pk, Bt, sl.p, tn, st);
    run_env_gemm(g1, prec, Rin.buf.p, Ri.rows, Ri.ld, sl.p, srows, ldS, t1b.p, err, st);
    if (tn == Num::F64) run_mix<double>(mx, t1b.as<double>(), t2b.p, tn, st);
    else run_mix<float>(mx, t1b.as<float>(), t2b.p, tn, st);
    run_env_gemm(g3, prec, t2b.p, trow, ldT, sl.p, srows, ldS, Rout.buf.p, err, st);
    Rout.op_valid = false;
    Rout.op32_valid = false;
    PD_CK(cudaStreamSynchronize(st));
}

// ------------------------------------------------------------------------------------------
// Two-site wavefunction from site tensors
// ------------------------------------------------------------------------------------------
void form_two_site(const Sec& bl, const Sec& bm, const Sec& br, const std::vector<int>& qn, const double* left,
                   const double* right, const double* mid, double* psi, cudaStream_t st) {
    const int d = (int)qn.size();
    const SiteLayout SL = site_layout(bl, bm, qn);
    const SiteLayout SR = site_layout(bm, br, qn);
    const PsiLayout P = psi_layout(bl, br, qn);
    DBuf scaled;
    const double* lsrc = left;
    if (mid) {
        // left' = left with its middle (column) index scaled by mid
        std::vector<long long> moff(bm.n() + 1, 0);
        for (int i = 0; i < bm.n(); ++i) moff[i + 1] = moff[i] + bm.m[i];
        std::vector<ColScaleJob> jobs;
        int mx = 1;
        for (const auto& b : SL.blk) {
            jobs.push_back({b.off, b.off, moff[b.j], b.rows, b.cols});
            mx = std::max(mx, b.rows * b.cols);
        }
        DBuf dj;
        upload(dj, jobs, st);
        scaled.ensure(std::max<long long>(1, SL.size) * 8, st);
        if (!jobs.empty()) {
            k_colscale<<<dim3(gridn(mx, 256), (unsigned)jobs.size()), 256, 0, st>>>(dj.as<ColScaleJob>(), left, mid,
                                                                                   scaled.as<double>());
            PD_LAUNCHED();
        }
        lsrc = scaled.as<double>();
        PD_CK(cudaStreamSynchronize(st));
    }
    GemmBatch g;
    for (const auto& b : P.blk) {
        int im = bm.find(bl.q[b.i] + qn[b.s1]);
        if (im < 0) continue;
        int lb = SL.at(b.i, b.s1), rb = SR.at(im, b.s2);
        if (lb < 0 || rb < 0) continue;
        // C(m = c, n = a) = sum_mid right[mid][c] left[a][mid]
        g.add(b.cols, b.rows, b.off, 1, b.cols, bm.m[im], 1, 1, b.cols,
              {GSeg{SR.blk[rb].off, SL.blk[lb].off, bm.m[im], 0}});
    }
    PD_CK(cudaMemsetAsync(psi, 0, sizeof(double) * std::max<long long>(1, P.size), st));
    (void)d;
    run_gemm64(g, right, lsrc, psi, st);
    PD_CK(cudaStreamSynchronize(st));
}

// ------------------------------------------------------------------------------------------
// SVD split with truncation (Eq. svd)
// ------------------------------------------------------------------------------------------
namespace {
struct SecInfo {
    int qm = 0;
    std::map<std::pair<int, int>, int> roff, coff;   // (i, s1) -> row offset, (s2, k) -> col offset
    int r = 0, c = 0;
};
std::map<int, SecInfo> split_sectors(const PsiLayout& P, const Sec& bl, const Sec& br, const std::vector<int>& qn1) {
    std::map<int, SecInfo> secs;
    for (const auto& b : P.blk) {
        int qm = bl.q[b.i] + qn1[b.s1];
        auto& S = secs[qm];
        S.qm = qm;
        S.roff[{b.i, b.s1}] = 0;
        S.coff[{b.s2, b.k}] = 0;
    }
    for (auto& kv : secs) {
        auto& S = kv.second;
        int o = 0;
        for (auto& r : S.roff) { r.second = o; o += bl.m[r.first.first]; }
        S.r = o;
        o = 0;
        for (auto& c : S.coff) { c.second = o; o += br.m[c.first.second]; }
        S.c = o;
    }
    return secs;
}
}  // namespace

void svd_split_bounds(const Sec& bl, const Sec& br, const std::vector<int>& qn1, const std::vector<int>& qn2,
                      long long* a_elems, long long* b_elems, long long* lam_elems) {
    const PsiLayout P = psi_layout2(bl, br, qn1, qn2);
    auto secs = split_sectors(P, bl, br, qn1);
    long long a = 0, b = 0, l = 0;
    for (auto& kv : secs) {
        long long k = std::min(kv.second.r, kv.second.c);
        a += (long long)kv.second.r * k;
        b += k * kv.second.c;
        l += k;
    }
    *a_elems = a;
    *b_elems = b;
    *lam_elems = l;
}

namespace {

// Column copy: dst[dst + r] = scale * src[src + r] for r < rows, scale = 1 / sig[sig_idx] (0 when
// that value is 0) if sig_idx >= 0, else 1.  One CTA per column.
struct ColJob {
    long long src, dst, sig_idx;
    int rows, pad_;
};
__global__ void k_col_copy(const ColJob* __restrict__ jobs, const double* __restrict__ src, double* __restrict__ dst,
                           const double* __restrict__ sig) {
    const ColJob j = jobs[blockIdx.x];
    double sc = 1.0;
    if (j.sig_idx >= 0) {
        const double v = sig[j.sig_idx];
        sc = v > 0.0 ? 1.0 / v : 0.0;
    }
    for (int r = threadIdx.x; r < j.rows; r += blockDim.x) dst[j.dst + r] = sc * src[j.src + r];
}

void col_copy(const std::vector<ColJob>& jobs, const double* src, double* dst, const double* sig, cudaStream_t st) {
    if (jobs.empty()) return;
    DBuf dj;
    upload(dj, jobs, st);
    k_col_copy<<<(unsigned)jobs.size(), 128, 0, st>>>(dj.as<ColJob>(), src, dst, sig);
    PD_LAUNCHED();
}

// FP64 one-sided Jacobi SVD of the column-major matrices W_s (p_s x n_s, n_s <= p_s) at ss[s].w_off
// of W (overwritten by U_s Sigma_s).  Fills v_off / s_off / npad / pair0 of ss; V receives V_s,
// sig the column norms and ord their descending order; dsecs the device copy of ss.
// FP32 block Jacobi (one task per block pair, n / 16 - 1 rounds per sweep) of the batch ss: W (p x n
// at w_off), rotations accumulated into V (n x n at v_off, initialised by the caller); rot: sweep
// histogram (max_sweeps + 1 ints, zeroed), bar: 3 zeroed barrier words, err: error word.
void block_jacobi32(const std::vector<SvdSec>& ss, const SvdSec* dsecs, float* W, float* V, int max_rows, int max_n,
                    int max_sweeps, int* rot, unsigned* bar, unsigned* err, unsigned long long* flops, cudaStream_t st) {
    const int nsec = (int)ss.size();
    std::vector<BjSec> bs(nsec);
    std::vector<int> task_sec;
    int nrounds = 0, nblk = 0, npst = 0;
    for (int s = 0; s < nsec; ++s) {
        BjSec b{};
        b.nb = (ss[s].n + 15) / 16;
        b.nbp = b.nb + (b.nb & 1);
        b.task0 = (int)task_sec.size();
        b.ntask = b.nb == 0 ? 0 : (b.nb == 1 ? 1 : b.nbp / 2);
        // each sector's own threshold, so a split's result does not depend on its batch
        b.tol = std::max(3e-5f, 16.0f * FLT_EPSILON * std::sqrt((float)std::max(1, ss[s].p)));
        b.blk0 = nblk;
        b.pst0 = npst;
        nblk += b.nb;
        npst += b.nb * b.nb;
        for (int t = 0; t < b.ntask; ++t) task_sec.push_back(s);
        if (b.nb > 0) nrounds = std::max(nrounds, b.nb == 1 ? 1 : b.nbp - 1);
        bs[s] = b;
    }
    // the dependency queue's items for one sweep: round by round, in each round the pairs of every
    // sector that has the round, taller sectors first (their pairs are the longest)
    std::vector<int> by_rows(nsec);
    for (int s = 0; s < nsec; ++s) by_rows[s] = s;
    std::stable_sort(by_rows.begin(), by_rows.end(), [&](int a, int b) { return ss[a].p > ss[b].p; });
    std::vector<int2> items;
    int nact = 0;
    for (const BjSec& b : bs) nact += b.nb > 0;
    for (int r = 0; r < nrounds; ++r)
        for (int s : by_rows) {
            const BjSec& b = bs[s];
            const int nr = b.nb == 0 ? 0 : (b.nb == 1 ? 1 : b.nbp - 1);
            if (r < nr)
                for (int t = 0; t < b.ntask; ++t) items.push_back(make_int2(s, (r << 16) | t));
        }
    const int bj_sweeps = std::min(40, max_sweeps);   // sweep cap of the block Jacobi
    PD_REQUIRE(nrounds < 32768 && (long long)items.size() * bj_sweeps < (1ll << 31), DMRG_ERR_CAPACITY,
               "block Jacobi: too many work items");
    DBuf dbs, dts, dgmax, dstamp, ditems, dq;
    upload(dbs, bs, st);
    upload(dts, task_sec, st);
    upload(ditems, items, st);
    const size_t nq = 3 + (size_t)nsec * (2 + bj_sweeps);
    dq.ensure(nq * 4, st);
    PD_CK(cudaMemsetAsync(dq.p, 0, nq * 4, st));
    dgmax.ensure(std::max(1, nsec) * 4, st);
    PD_CK(cudaMemsetAsync(dgmax.p, 0, std::max(1, nsec) * 4, st));
    // block / pair stamps (zero: never rotated / never found converged)
    dstamp.ensure((size_t)std::max(1, nblk + npst) * 4, st);
    PD_CK(cudaMemsetAsync(dstamp.p, 0, (size_t)std::max(1, nblk + npst) * 4, st));
    PD_CK(cudaMemsetAsync(flops, 0, 8, st));
    launch_bjacobi(dsecs, dbs.as<BjSec>(), dts.as<int>(), (int)task_sec.size(), nrounds, max_rows, max_n, bj_sweeps, 2,
                   W, V, 8.0f * FLT_EPSILON, dgmax.as<float>(), dstamp.as<int>(), dstamp.as<int>() + nblk, rot,
                   rot + max_sweeps, bar, err, flops, ditems.as<int2>(), (int)items.size(), nsec, nact, dq.as<int>(), st);
}

// Preconditioning of an FP64 one-sided Jacobi SVD of the batch ss (W FP64, p x n at w_off): the FP32
// block Jacobi on an FP32 copy, its rotations orthonormalised in FP64 (Newton-Schulz) into V
// (n x n at v_off), and W <- W V in FP64.  The FP64 Jacobi then starts from V with columns that are
// orthogonal to FP32 accuracy, so its sweeps converge in the quadratic regime.
void fp64_precondition(const std::vector<SvdSec>& ss, const SvdSec* dsecs, DBuf& dW, double* V, long long woff,
                       long long voff, int maxp, int maxn, unsigned* bar, unsigned* err, cudaStream_t st) {
    const int max_sweeps = 60;
    DBuf w32, v32, rot32, fl, dW1;
    w32.ensure(woff * 4, st);
    v32.ensure(std::max<long long>(1, voff) * 4, st);
    rot32.ensure((max_sweeps + 1) * 4, st);
    fl.ensure(8, st);
    PD_CK(cudaMemsetAsync(rot32.p, 0, (max_sweeps + 1) * 4, st));
    PD_CK(cudaMemsetAsync(bar, 0, 3 * sizeof(unsigned), st));
    convert_flat(dW.p, Num::F64, w32.p, Num::F32, woff, st);
    launch_svd_init_v<float>(dsecs, (int)ss.size(), maxn, v32.as<float>(), st);
    block_jacobi32(ss, dsecs, w32.as<float>(), v32.as<float>(), maxp, maxn, max_sweeps, rot32.as<int>(), bar, err,
                   fl.as<unsigned long long>(), st);
    convert_flat(v32.p, Num::F32, V, Num::F64, voff, st);
    orthonormalize_square(ss, V, st);
    GemmBatch gwq;
    for (const auto& x : ss)
        if (x.n > 0)   // W1(r, c) = sum_u W(r, u) V(u, c)
            gwq.add(x.p, x.n, x.w_off, 1, x.p, x.n, 1, 1, x.p, {GSeg{x.w_off, x.v_off, x.n, 0}});
    dW1.ensure(woff * 8, st);
    run_gemm64(gwq, dW.as<double>(), V, dW1.as<double>(), st);
    PD_CK(cudaMemsetAsync(bar, 0, 3 * sizeof(unsigned), st));
    dW = std::move(dW1);
}

void jacobi64(std::vector<SvdSec>& ss, DBuf& dWbuf, DBuf& dsecs, DBuf& dV, DBuf& dsig, DBuf& dord, cudaStream_t st) {
    const int nsec = (int)ss.size();
    std::vector<int> pair_sec;
    long long voff = 0, soff = 0;
    int maxn = 0, maxnpad = 0, maxp = 1;
    for (int s = 0; s < nsec; ++s) {
        SvdSec& x = ss[s];
        x.npad = x.n + (x.n & 1);
        x.v_off = voff;
        x.s_off = soff;
        x.pair0 = (int)pair_sec.size();
        for (int i = 0; i < x.npad / 2; ++i) pair_sec.push_back(s);
        voff += (long long)x.n * x.n;
        soff += x.n;
        maxn = std::max(maxn, x.n);
        maxp = std::max(maxp, x.p);
        maxnpad = std::max(maxnpad, x.npad);
    }
    const int max_sweeps = 60;
    DBuf dpairs, drot, dbar;
    upload(dsecs, ss, st);
    upload(dpairs, pair_sec, st);
    dV.ensure(std::max<long long>(1, voff) * 8, st);
    dsig.ensure(std::max<long long>(1, soff) * 8, st);
    dord.ensure(std::max<long long>(1, soff) * 4, st);
    drot.ensure((max_sweeps + 1) * 4, st);
    dbar.ensure(4 * sizeof(unsigned), st);
    PD_CK(cudaMemsetAsync(drot.p, 0, (max_sweeps + 1) * 4, st));
    PD_CK(cudaMemsetAsync(dbar.p, 0, 4 * sizeof(unsigned), st));
    unsigned* bar = dbar.as<unsigned>();
    const long long woff = ss.empty() ? 0 : ss.back().w_off + (long long)ss.back().p * ss.back().n;
    if (g_svd_qr && woff > 0)
        fp64_precondition(ss, dsecs.as<SvdSec>(), dWbuf, dV.as<double>(), woff, voff, maxp, maxn, bar, bar + 3, st);
    else
        launch_svd_init_v<double>(dsecs.as<SvdSec>(), nsec, maxn, dV.as<double>(), st);
    double* W = dWbuf.as<double>();
    const double tol = 4.0 * DBL_EPSILON;
    launch_jacobi<double>(dsecs.as<SvdSec>(), nsec, dpairs.as<int>(), (int)pair_sec.size(), maxnpad, max_sweeps, W,
                          dV.as<double>(), tol, 0.0, nullptr, drot.as<int>(), drot.as<int>() + max_sweeps, bar, bar + 3,
                          st);
    launch_svd_finish<double>(dsecs.as<SvdSec>(), nsec, W, dsig.as<double>(), dord.as<int>(), st);
    unsigned err = 0;
    PD_CK(cudaMemcpyAsync(&err, bar + 3, 4, cudaMemcpyDeviceToHost, st));
    PD_CK(cudaStreamSynchronize(st));
    PD_REQUIRE(!(err & ERRBIT_TIMEOUT), DMRG_ERR_TIMEOUT, "Jacobi SVD grid barrier timed out");
}

// The Appendix's accurate SVD, applied to a finished batch (W = U Sigma, V, sig, ord; M the
// matrices the SVD was taken of, same layout as W).  Per matrix, with singular values
// lambda_1 >= ... >= lambda_n: p = the first index with lambda_p / lambda_1 < eps; if there is one,
// X = U_p^T M V_p over the columns p..n, the same SVD and refinement recursively on X, then
// U_p <- U_p U_X, V_p <- V_p V_X, lambda_p.. <- lambda_X.  Results written back into W, V, and
// sig / ord recomputed.
constexpr double ACC_EPS = 1e-4;
void accurate_refine(const std::vector<SvdSec>& ss, const SvdSec* dsecs, double* W, double* V, double* sig, int* ord,
                     const double* M, int depth, cudaStream_t st) {
    const int nsec = (int)ss.size();
    long long total = 0;
    for (const auto& x : ss) total = std::max(total, x.s_off + x.n);
    if (total == 0) return;
    std::vector<double> hsig(total);
    std::vector<int> hord(total);
    PD_CK(cudaMemcpyAsync(hsig.data(), sig, total * 8, cudaMemcpyDeviceToHost, st));
    PD_CK(cudaMemcpyAsync(hord.data(), ord, total * 4, cudaMemcpyDeviceToHost, st));
    PD_CK(cudaStreamSynchronize(st));
    struct Ref {
        int s, p, q;
        long long up, vp, x;
    };
    std::vector<Ref> refs;
    long long nup = 0, nvp = 0, nx = 0;
    for (int s = 0; s < nsec; ++s) {
        const SvdSec& S = ss[s];
        if (S.n <= 1) continue;
        const double l0 = hsig[S.s_off + hord[S.s_off]];
        if (!(l0 > 0.0)) continue;
        int p = -1;
        for (int i = 1; i < S.n; ++i)
            if (hsig[S.s_off + hord[S.s_off + i]] / l0 < ACC_EPS) {
                p = i;
                break;
            }
        if (p < 0) continue;
        const int q = S.n - p;
        refs.push_back({s, p, q, nup, nvp, nx});
        nup += (long long)S.p * q;
        nvp += (long long)S.n * q;
        nx += (long long)q * q;
    }
    if (refs.empty()) return;
    PD_REQUIRE(depth < 64, DMRG_ERR_NUMERIC, "accurate SVD recursion did not terminate");
    DBuf dUp, dVp, dT, dX;
    dUp.ensure(nup * 8, st);
    dVp.ensure(nvp * 8, st);
    dT.ensure(nup * 8, st);
    dX.ensure(nx * 8, st);
    // U_p (normalised columns of W in descending order from p) and V_p
    std::vector<ColJob> gu, gv;
    for (const auto& r : refs) {
        const SvdSec& S = ss[r.s];
        for (int j = 0; j < r.q; ++j) {
            const int c = hord[S.s_off + r.p + j];
            gu.push_back({S.w_off + (long long)c * S.p, r.up + (long long)j * S.p, S.s_off + c, S.p, 0});
            gv.push_back({S.v_off + (long long)c * S.n, r.vp + (long long)j * S.n, -1, S.n, 0});
        }
    }
    col_copy(gu, W, dUp.as<double>(), sig, st);
    col_copy(gv, V, dVp.as<double>(), nullptr, st);
    // T = M V_p (p x q), X = U_p^T T (q x q)
    GemmBatch g1, g2;
    for (const auto& r : refs) {
        const SvdSec& S = ss[r.s];
        g1.add(S.p, r.q, r.up, 1, S.p, S.n, 1, 1, S.p, {GSeg{S.w_off, r.vp, S.n, 0}});
        g2.add(r.q, r.q, r.x, S.p, 1, S.p, 1, 1, r.q, {GSeg{r.up, r.up, S.p, 0}});
    }
    run_gemm64(g1, M, dVp.as<double>(), dT.as<double>(), st);
    run_gemm64(g2, dUp.as<double>(), dT.as<double>(), dX.as<double>(), st);
    // the same SVD and refinement of X
    std::vector<SvdSec> xs(refs.size());
    for (size_t i = 0; i < refs.size(); ++i) {
        xs[i] = SvdSec{};
        xs[i].w_off = refs[i].x;
        xs[i].p = xs[i].n = refs[i].q;
    }
    DBuf dXW, dXsecs, dXV, dXsig, dXord;
    dXW.ensure(nx * 8, st);
    PD_CK(cudaMemcpyAsync(dXW.p, dX.p, nx * 8, cudaMemcpyDeviceToDevice, st));
    jacobi64(xs, dXW, dXsecs, dXV, dXsig, dXord, st);
    accurate_refine(xs, dXsecs.as<SvdSec>(), dXW.as<double>(), dXV.as<double>(), dXsig.as<double>(),
                    dXord.as<int>(), dX.as<double>(), depth + 1, st);
    std::vector<int> hxo(nx > 0 ? (size_t)std::max<long long>(1, xs.back().s_off + xs.back().n) : 1);
    PD_CK(cudaMemcpyAsync(hxo.data(), dXord.p, hxo.size() * 4, cudaMemcpyDeviceToHost, st));
    PD_CK(cudaStreamSynchronize(st));
    // X factors with columns in descending order (W_X keeps U_X Sigma_X)
    DBuf dWxp, dVxp;
    dWxp.ensure(nx * 8, st);
    dVxp.ensure(nx * 8, st);
    std::vector<ColJob> gw, gx;
    for (size_t i = 0; i < refs.size(); ++i) {
        const int q = refs[i].q;
        for (int j = 0; j < q; ++j) {
            const int c = hxo[xs[i].s_off + j];
            gw.push_back({xs[i].w_off + (long long)c * q, refs[i].x + (long long)j * q, -1, q, 0});
            gx.push_back({xs[i].v_off + (long long)c * q, refs[i].x + (long long)j * q, -1, q, 0});
        }
    }
    col_copy(gw, dXW.as<double>(), dWxp.as<double>(), nullptr, st);
    col_copy(gx, dXV.as<double>(), dVxp.as<double>(), nullptr, st);
    // new columns: U_p (U_X Sigma_X) into T, V_p V_X into Vn
    DBuf dVn;
    dVn.ensure(nvp * 8, st);
    GemmBatch g3, g4;
    for (const auto& r : refs) {
        const SvdSec& S = ss[r.s];
        g3.add(S.p, r.q, r.up, 1, S.p, r.q, 1, 1, S.p, {GSeg{r.up, r.x, r.q, 0}});
        g4.add(S.n, r.q, r.vp, 1, S.n, r.q, 1, 1, S.n, {GSeg{r.vp, r.x, r.q, 0}});
    }
    run_gemm64(g3, dUp.as<double>(), dWxp.as<double>(), dT.as<double>(), st);
    run_gemm64(g4, dVp.as<double>(), dVxp.as<double>(), dVn.as<double>(), st);
    std::vector<ColJob> sw, sv;
    for (const auto& r : refs) {
        const SvdSec& S = ss[r.s];
        for (int j = 0; j < r.q; ++j) {
            const int c = hord[S.s_off + r.p + j];
            sw.push_back({r.up + (long long)j * S.p, S.w_off + (long long)c * S.p, -1, S.p, 0});
            sv.push_back({r.vp + (long long)j * S.n, S.v_off + (long long)c * S.n, -1, S.n, 0});
        }
    }
    col_copy(sw, dT.as<double>(), W, nullptr, st);
    col_copy(sv, dVn.as<double>(), V, nullptr, st);
    launch_svd_finish<double>(dsecs, nsec, W, sig, ord, st);
}

}  // namespace

std::vector<SplitResult> svd_split_batch(const std::vector<SplitReq>& reqs, bool accurate, bool fp32, cudaStream_t st) {
    const size_t es = fp32 ? 4 : 8;
    const int nreq = (int)reqs.size();
    // per bond: sector layout (rows (i, s1) sorted, cols (s2, k) sorted, per middle charge); the
    // sectors of all bonds are numbered consecutively and packed into joint W / V / sigma buffers
    struct Front {
        PsiLayout P;
        std::map<int, SecInfo> secs;
        std::vector<SecInfo*> order;
        int sec0 = 0, nsec = 0, total = 0, maxp = 1;
        long long sbase = 0;
    };
    std::vector<Front> fr(nreq);
    std::vector<SvdSec> ss;
    std::vector<int> pair_sec;
    long long woff = 0, voff = 0, soff = 0;
    int maxn = 0, maxnpad = 0, maxp = 1, max_total = 1, max_nsec = 1;
    for (int q = 0; q < nreq; ++q) {
        const SplitReq& R = reqs[q];
        Front& F = fr[q];
        F.P = psi_layout2(R.bl, R.br, *R.qn1, *R.qn2);
        F.secs = split_sectors(F.P, R.bl, R.br, *R.qn1);
        for (auto& kv : F.secs) F.order.push_back(&kv.second);
        F.sec0 = (int)ss.size();
        F.nsec = (int)F.order.size();
        F.sbase = soff;
        for (int s = 0; s < F.nsec; ++s) {
            const auto& S = *F.order[s];
            SvdSec x{};
            x.p = std::max(S.r, S.c);
            x.n = std::min(S.r, S.c);
            x.npad = x.n + (x.n & 1);
            x.w_off = woff; x.v_off = voff; x.s_off = soff;
            x.pair0 = (int)pair_sec.size();
            for (int i = 0; i < x.npad / 2; ++i) pair_sec.push_back(F.sec0 + s);
            woff += (long long)x.p * x.n;
            voff += (long long)x.n * x.n;
            soff += x.n;
            maxn = std::max(maxn, x.n);
            F.maxp = std::max(F.maxp, x.p);
            maxnpad = std::max(maxnpad, x.npad);
            ss.push_back(x);
        }
        F.total = (int)(soff - F.sbase);
        maxp = std::max(maxp, F.maxp);
        max_total = std::max(max_total, F.total);
        max_nsec = std::max(max_nsec, F.nsec);
    }
    const int nsec = (int)ss.size();
    // gather each bond's Psi blocks into its matrices (W = M, or M^T when M is wide; column-major)
    std::vector<CopyList> gather(nreq);
    for (int q = 0; q < nreq; ++q) {
        const Front& F = fr[q];
        const std::vector<int>& qn = *reqs[q].qn1;
        for (const auto& b : F.P.blk) {
            const int qm = reqs[q].bl.q[b.i] + qn[b.s1];
            const int s = (int)(std::find_if(F.order.begin(), F.order.end(), [&](SecInfo* x) { return x->qm == qm; }) -
                                F.order.begin());
            const auto& S = *F.order[s];
            const SvdSec& x = ss[F.sec0 + s];
            const int r0 = S.roff.at({b.i, b.s1}), c0 = S.coff.at({b.s2, b.k});
            CopyJob j{};
            j.src = b.off; j.rows = b.rows; j.cols = b.cols; j.srs = b.cols; j.scs = 1; j.zero_to = 0; j.scale = 1.0;
            if (S.r >= S.c) {
                j.dst = x.w_off + (long long)c0 * S.r + r0; j.drs = 1; j.dcs = S.r;
            } else {
                j.dst = x.w_off + (long long)r0 * S.c + c0; j.drs = S.c; j.dcs = 1;
            }
            gather[q].add(j);
        }
    }
    DBuf dW, dV, dsig, dord, dsecs, dpairs, drot, dkept, dwts, dbar, dflops;
    dflops.ensure(8, st);
    const int max_sweeps = 60;
    dbar.ensure(4 * sizeof(unsigned), st);     // barrier words + the error word
    PD_CK(cudaMemsetAsync(dbar.p, 0, 4 * sizeof(unsigned), st));
    unsigned* bar = dbar.as<unsigned>();
    unsigned* jerr = bar + 3;
    dW.ensure(std::max<long long>(1, woff) * es, st);
    dV.ensure(std::max<long long>(1, voff) * es, st);
    dsig.ensure(std::max<long long>(1, soff) * 8, st);
    dord.ensure(std::max<long long>(1, soff) * 4, st);
    dkept.ensure(std::max(1, nsec) * 4, st);
    dwts.ensure(std::max(1, nreq) * 16, st);
    drot.ensure((max_sweeps + 1) * 4, st);
    upload(dsecs, ss, st);
    upload(dpairs, pair_sec, st);
    for (auto& g : gather) g.up(st);
    PD_CK(cudaMemsetAsync(dW.p, 0, std::max<long long>(1, woff) * es, st));
    PD_CK(cudaMemsetAsync(drot.p, 0, (max_sweeps + 1) * 4, st));
    const int npairs = (int)pair_sec.size();
    cudaEvent_t sv0 = nullptr, sv1 = nullptr;
    if (prof_on()) {
        PD_CK(cudaEventCreate(&sv0));
        PD_CK(cudaEventCreate(&sv1));
        PD_CK(cudaEventRecord(sv0, st));
    }
    // QR preconditioning: the Jacobi runs on X = R^T (n x n per sector, stored at v_off of dV) with
    // its rotations accumulated in dVJ; afterwards dW receives Q [V_J Sigma; 0] and dV the right
    // singular vectors -- the same outputs as the plain Jacobi on W.
    QrPlan qp;
    DBuf dxsecs, dVJ;
    std::vector<SvdSec> xs;
    if (g_svd_qr && woff > 0 && fp32) {
        qp.build<float>(ss, st);
        if (qp.ok) {
            xs = ss;
            for (auto& x : xs) {
                x.w_off = x.v_off;
                x.p = x.n;
            }
            upload(dxsecs, xs, st);
            dVJ.ensure(std::max<long long>(1, voff) * es, st);
        }
    }
    const bool use_qr = qp.ok && !xs.empty();
    const SvdSec* jsecs = use_qr ? dxsecs.as<SvdSec>() : dsecs.as<SvdSec>();
    const int jmaxp = use_qr ? maxn : maxp;
    if (fp32) {
        for (int q = 0; q < nreq; ++q) run_copy<double>(gather[q], reqs[q].psi, dW.p, Num::F32, st);
        float* JW = dW.as<float>();
        float* JV = dV.as<float>();
        if (use_qr) {
            qp.factor<float>(dW.as<float>(), st);
            qp.form_rt<float>(dW.as<float>(), dV.as<float>(), st);
            JW = dV.as<float>();
            JV = dVJ.as<float>();
        }
        launch_svd_init_v<float>(jsecs, nsec, maxn, JV, st);
        // the kept factor that joins a block is re-orthonormalised in FP64 afterwards
        block_jacobi32(use_qr ? xs : ss, jsecs, JW, JV, jmaxp, maxn, max_sweeps, drot.as<int>(), bar, jerr,
                       dflops.as<unsigned long long>(), st);
        if (use_qr) {
            DBuf dWo;
            dWo.ensure(std::max<long long>(1, woff) * es, st);
            qp.finish<float>(dW.as<float>(), dV.as<float>(), dVJ.as<float>(), dWo.as<float>(), st);
            dW = std::move(dWo);
        }
        launch_svd_finish<float>(dsecs.as<SvdSec>(), nsec, dW.as<float>(), dsig.as<double>(), dord.as<int>(), st);
    } else {
        for (int q = 0; q < nreq; ++q) run_copy<double>(gather[q], reqs[q].psi, dW.p, Num::F64, st);
        DBuf dM;
        if (accurate && woff > 0) {
            dM.ensure(woff * 8, st);
            PD_CK(cudaMemcpyAsync(dM.p, dW.p, woff * 8, cudaMemcpyDeviceToDevice, st));
        }
        const double tol = 4.0 * DBL_EPSILON;   // per sector: times sqrt(p)
        if (g_svd_qr && woff > 0)
            fp64_precondition(ss, dsecs.as<SvdSec>(), dW, dV.as<double>(), woff, voff, maxp, maxn, bar, jerr, st);
        else
            launch_svd_init_v<double>(dsecs.as<SvdSec>(), nsec, maxn, dV.as<double>(), st);
        launch_jacobi<double>(dsecs.as<SvdSec>(), nsec, dpairs.as<int>(), npairs, maxnpad, max_sweeps, dW.as<double>(),
                              dV.as<double>(), tol, 0.0, nullptr, drot.as<int>(), drot.as<int>() + max_sweeps, bar, jerr,
                              st);
        launch_svd_finish<double>(dsecs.as<SvdSec>(), nsec, dW.as<double>(), dsig.as<double>(), dord.as<int>(), st);
        if (accurate && woff > 0)
            accurate_refine(ss, dsecs.as<SvdSec>(), dW.as<double>(), dV.as<double>(), dsig.as<double>(),
                            dord.as<int>(), dM.as<double>(), 0, st);
    }
    if (sv0) {
        PD_CK(cudaEventRecord(sv1, st));
        int sweeps = 0;
        unsigned long long fl = 0;
        std::vector<int> hist(max_sweeps, 0);
        PD_CK(cudaMemcpyAsync(&sweeps, drot.as<int>() + max_sweeps, 4, cudaMemcpyDeviceToHost, st));
        PD_CK(cudaMemcpyAsync(hist.data(), drot.p, 4 * max_sweeps, cudaMemcpyDeviceToHost, st));
        if (fp32) PD_CK(cudaMemcpyAsync(&fl, dflops.p, 8, cudaMemcpyDeviceToHost, st));
        PD_CK(cudaStreamSynchronize(st));
        float ms = 0.f;
        PD_CK(cudaEventElapsedTime(&ms, sv0, sv1));
        double alg_fl = 0.0, alg_b = 0.0;
        for (const SvdSec& x : ss) {
            const double p = x.p, n = x.n;
            alg_fl += 4.0 * p * n * n + 22.0 * n * n * n;
            alg_b += 4.0 * (2.0 * p * n + n * n);
        }
        prof_svd(sweeps, ms, fp32 ? 1 : 2, maxp, (double)fl, fp32 ? hist.data() : nullptr, max_sweeps, nreq, alg_fl,
                 alg_b);
        cudaEventDestroy(sv0);
        cudaEventDestroy(sv1);
    }
    // truncation per bond (the keep-m rule runs over one bond's sectors): its sector table with
    // sigma offsets relative to the bond's first sector, and sigma / order shifted to match
    std::vector<SvdSec> tl = ss;
    for (const Front& F : fr)
        for (int s = 0; s < F.nsec; ++s) tl[F.sec0 + s].s_off -= F.sbase;
    DBuf dtl, tsd, tsi;
    upload(dtl, tl, st);
    tsd.ensure((size_t)(max_total + max_nsec + 1) * 8, st);
    tsi.ensure((size_t)(3 * max_total + 1) * 4, st);
    // an FP32 SVD reports exact zeros at ~1e-7 of the largest singular value: keep its cutoff
    // above that noise floor (the discarded weight stays below 1e-10)
    for (int q = 0; q < nreq; ++q) {
        const Front& F = fr[q];
        const double cutoff = fp32 ? std::max(reqs[q].rel_cutoff, 1e-5) : reqs[q].rel_cutoff;
        launch_truncate(dtl.as<SvdSec>() + F.sec0, F.nsec, dsig.as<double>() + F.sbase, dord.as<int>() + F.sbase,
                        F.total, reqs[q].m_max, cutoff, 1e-10, dkept.as<int>() + F.sec0, dwts.as<double>() + 2 * q,
                        tsd.as<double>(), tsi.as<int>(), st);
    }
    std::vector<int> kept(std::max(1, nsec));
    std::vector<double> wts(2 * std::max(1, nreq));
    unsigned jerr_h = 0;
    int sweeps_h = 0;
    PD_CK(cudaMemcpyAsync(&sweeps_h, drot.as<int>() + max_sweeps, 4, cudaMemcpyDeviceToHost, st));
    PD_CK(cudaMemcpyAsync(&jerr_h, jerr, 4, cudaMemcpyDeviceToHost, st));
    PD_CK(cudaMemcpyAsync(kept.data(), dkept.p, 4 * std::max(1, nsec), cudaMemcpyDeviceToHost, st));
    PD_CK(cudaMemcpyAsync(wts.data(), dwts.p, 16 * std::max(1, nreq), cudaMemcpyDeviceToHost, st));
    PD_CK(cudaStreamSynchronize(st));
    PD_REQUIRE(!(jerr_h & ERRBIT_TIMEOUT), DMRG_ERR_TIMEOUT, "Jacobi SVD grid barrier timed out");
    std::vector<SplitResult> out(nreq);
    std::vector<DBuf> keep_alive;
    keep_alive.reserve(4 * nreq);
    for (int q = 0; q < nreq; ++q) {
        const Front& F = fr[q];
        const SplitReq& R = reqs[q];
        const std::vector<int>& qn1 = *R.qn1;
        const std::vector<int>& qn2 = *R.qn2;
        SplitResult& res = out[q];
        res.sweeps = sweeps_h;
        res.max_rows = F.maxp;
        std::vector<int> kept_of_sec(F.nsec, 0);
        for (int s = 0; s < F.nsec; ++s)
            if (kept[F.sec0 + s] > 0) {
                res.mid.q.push_back(F.order[s]->qm);
                res.mid.m.push_back(kept[F.sec0 + s]);
                kept_of_sec[s] = kept[F.sec0 + s];
            }
        PD_REQUIRE(res.mid.n() > 0, DMRG_ERR_NUMERIC, "SVD kept no singular value (zero wavefunction?)");
        const double w0 = wts[2 * q], w1 = wts[2 * q + 1];
        res.trunc = w0 > 0 ? std::max(0.0, (w0 - w1) / w0) : 0.0;
        // scatter
        const SiteLayout SA = site_layout(R.bl, res.mid, qn1);
        const SiteLayout SB = site_layout(res.mid, R.br, qn2);
        std::vector<ScatJob> ja, jb;
        int mx = 1;
        for (int s = 0; s < F.nsec; ++s) {
            if (!kept_of_sec[s]) continue;
            const auto& S = *F.order[s];
            const SvdSec& x = ss[F.sec0 + s];
            const int im = res.mid.find(S.qm);
            const bool rge = S.r >= S.c;
            for (const auto& r : S.roff) {        // A blocks (i, s1) [a][k]
                const int ab = SA.at(r.first.first, r.first.second);
                if (ab < 0) continue;
                ScatJob j{};
                j.dst = SA.blk[ab].off; j.rows = SA.blk[ab].rows; j.cols = SA.blk[ab].cols;
                j.s_off = x.s_off; j.off0 = r.second; j.left = 1; j.lam_pow = R.lam_pow_left;
                if (rge) { j.fromW = 1; j.base = x.w_off; j.ld = x.p; }
                else { j.fromW = 0; j.base = x.v_off; j.ld = x.n; }
                ja.push_back(j);
                mx = std::max(mx, j.rows * j.cols);
            }
            for (const auto& c : S.coff) {        // B blocks (m, s2) [k][c]
                const int bb = SB.at(im, c.first.first);
                if (bb < 0) continue;
                ScatJob j{};
                j.dst = SB.blk[bb].off; j.rows = SB.blk[bb].rows; j.cols = SB.blk[bb].cols;
                j.s_off = x.s_off; j.off0 = c.second; j.left = 0; j.lam_pow = R.lam_pow_right;
                if (rge) { j.fromW = 0; j.base = x.v_off; j.ld = x.n; }
                else { j.fromW = 1; j.base = x.w_off; j.ld = x.p; }
                jb.push_back(j);
                mx = std::max(mx, j.rows * j.cols);
            }
        }
        const double* wq = dwts.as<double>() + 2 * q;
        auto scatter = [&](const std::vector<ScatJob>& jobs_, double* dst) {
            if (jobs_.empty()) return;
            keep_alive.emplace_back();
            DBuf& dj = keep_alive.back();
            upload(dj, jobs_, st);
            dim3 g(gridn(mx, 256), (unsigned)jobs_.size());
            if (fp32)
                k_svd_scatter<float><<<g, 256, 0, st>>>(dj.as<ScatJob>(), dW.as<float>(), dV.as<float>(),
                                                        dsig.as<double>(), dord.as<int>(), wq, dst);
            else
                k_svd_scatter<double><<<g, 256, 0, st>>>(dj.as<ScatJob>(), dW.as<double>(), dV.as<double>(),
                                                         dsig.as<double>(), dord.as<int>(), wq, dst);
            PD_LAUNCHED();
        };
        scatter(ja, R.A_out);
        scatter(jb, R.B_out);
        // lambda
        std::vector<LamJob> lj;
        long long o = 0;
        for (int s = 0; s < F.nsec; ++s) {
            if (!kept_of_sec[s]) continue;
            lj.push_back({ss[F.sec0 + s].s_off, o, kept_of_sec[s], 0});
            o += kept_of_sec[s];
        }
        keep_alive.emplace_back();
        DBuf& dlj = keep_alive.back();
        upload(dlj, lj, st);
        double* lam_dev = R.lam_out_dev;
        if (!lam_dev) {
            keep_alive.emplace_back();
            DBuf& dlam = keep_alive.back();
            dlam.ensure(o * 8, st);
            lam_dev = dlam.as<double>();
        }
        k_lam_out<<<std::max<int>(1, (int)lj.size()), 128, 0, st>>>(dlj.as<LamJob>(), (int)lj.size(),
                                                                     dsig.as<double>(), dord.as<int>(), wq, lam_dev);
        PD_LAUNCHED();
        res.lam.resize(o);
        PD_CK(cudaMemcpyAsync(res.lam.data(), lam_dev, o * 8, cudaMemcpyDeviceToHost, st));
    }
    PD_CK(cudaStreamSynchronize(st));
    return out;
}

SplitResult svd_split(const Sec& bl, const Sec& br, const std::vector<int>& qn1, const std::vector<int>& qn2,
                      const double* psi, int m_max, double rel_cutoff, bool accurate, int lam_pow_left,
                      int lam_pow_right, double* A_out, double* B_out, double* lam_out_dev, cudaStream_t st,
                      bool fp32) {
    SplitReq r;
    r.bl = bl;
    r.br = br;
    r.qn1 = &qn1;
    r.qn2 = &qn2;
    r.psi = psi;
    r.m_max = m_max;
    r.rel_cutoff = rel_cutoff;
    r.lam_pow_left = lam_pow_left;
    r.lam_pow_right = lam_pow_right;
    r.A_out = A_out;
    r.B_out = B_out;
    r.lam_out_dev = lam_out_dev;
    return std::move(svd_split_batch({r}, accurate, fp32, st)[0]);
}

// ------------------------------------------------------------------------------------------
// Davidson (the Sec. II local eigensolver), FP64 vectors, same algorithm as the CPU oracle
// ------------------------------------------------------------------------------------------
DavResult davidson(HeffPlan& P, const EnvSlab& L, const EnvSlab& R, double* x, int kmax, double tol,
                   int max_iter, unsigned* err, cudaStream_t st, HeffPlan* acc, int refine_iters) {
    const long long n = P.psi.size;
    PD_REQUIRE(kmax >= 2 && kmax <= 32, DMRG_ERR_ARG, "Davidson kmax must be in [2, 32]");
    DavResult res;
    const int nch = (int)std::max<long long>(1, std::min<long long>(512, (n + 4095) / 4096));
    DBuf dV, dAV, dG, dyth, dpart, dd1, dd2, dnrm, du, dAu, dr, dt, ddg;
    dV.ensure((size_t)kmax * n * 8, st);
    dAV.ensure((size_t)kmax * n * 8, st);
    dG.ensure((size_t)kmax * kmax * 8, st);
    dyth.ensure((kmax + 1) * 8, st);
    dpart.ensure((size_t)std::max(2, kmax) * nch * 8, st);
    dd1.ensure((kmax + 1) * 8, st);
    dd2.ensure((kmax + 1) * 8, st);
    dnrm.ensure(4 * 8, st);
    du.ensure(n * 8, st);
    dAu.ensure(n * 8, st);
    dr.ensure(n * 8, st);
    dt.ensure(n * 8, st);
    ddg.ensure(n * 8, st);
    double* V = dV.as<double>();
    double* AV = dAV.as<double>();
    double* G = dG.as<double>();
    cudaEvent_t e0, e1;
    PD_CK(cudaEventCreate(&e0));
    PD_CK(cudaEventCreate(&e1));
    HeffPlan* cur = &P;
    auto mv = [&](const double* in, double* out) {
        PD_CK(cudaEventRecord(e0, st));
        heff_apply(*cur, L, R, in, out, err, st);
        PD_CK(cudaEventRecord(e1, st));
        PD_CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        PD_CK(cudaEventElapsedTime(&ms, e0, e1));
        if (cur == &P) {
            res.mv_ms += ms;
            res.matvecs++;
        } else {
            res.acc_ms += ms;
            res.acc_matvecs++;
        }
    };
    heff_diag(P, L, R, ddg.as<double>(), st);
    double hn[4];
    // one Davidson run from the normalised vector in x; leaves the Ritz vector in du (|u|^2 in dnrm[1])
    auto run = [&](int iters) {
        launch_nrm2(x, n, dpart.as<double>(), nch, dnrm.as<double>(), st);
        launch_scale(x, dnrm.as<double>(), n, V, 1, st);
        mv(V, AV);
        int k = 1;
        launch_dots(V, n, 1, AV, n, dpart.as<double>(), nch, dd1.as<double>(), st);
        k_place<<<1, 32, 0, st>>>(G, kmax, 0, dd1.as<double>(), dd1.as<double>());
        PD_LAUNCHED();
        for (int it = 1; it <= iters; ++it) {
            res.iters++;
            launch_small_eig(G, k, kmax, dyth.as<double>(), st);
            launch_ritz(V, AV, n, k, dyth.as<double>(), n, du.as<double>(), dAu.as<double>(), dr.as<double>(),
                        dpart.as<double>(), nch, dnrm.as<double>(), st);
            PD_CK(cudaMemcpyAsync(hn, dnrm.p, 16, cudaMemcpyDeviceToHost, st));
            PD_CK(cudaMemcpyAsync(hn + 2, dyth.p, 8, cudaMemcpyDeviceToHost, st));
            PD_CK(cudaStreamSynchronize(st));
            res.theta = hn[2];
            res.rnorm = std::sqrt(std::max(0.0, hn[0]));
            PD_REQUIRE(std::isfinite(res.theta) && std::isfinite(res.rnorm), DMRG_ERR_NUMERIC,
                       "non-finite Ritz value in Davidson");
            if (res.rnorm <= tol * std::max(1.0, std::fabs(res.theta)) || it == iters) break;
            launch_precond(dr.as<double>(), ddg.as<double>(), dyth.as<double>(), 1e-4, n, dt.as<double>(), st);
            if (k >= kmax) {   // restart from the Ritz vector
                launch_scale(du.as<double>(), dnrm.as<double>() + 1, n, V, 1, st);
                launch_scale(dAu.as<double>(), dnrm.as<double>() + 1, n, AV, 1, st);
                k = 1;
                launch_dots(V, n, 1, AV, n, dpart.as<double>(), nch, dd1.as<double>(), st);
                k_place<<<1, 32, 0, st>>>(G, kmax, 0, dd1.as<double>(), dd1.as<double>());
                PD_LAUNCHED();
            }
            for (int pass = 0; pass < 2; ++pass) {
                launch_dots(V, n, k, dt.as<double>(), n, dpart.as<double>(), nch, dd1.as<double>(), st);
                launch_subtract(V, n, k, dd1.as<double>(), n, dt.as<double>(), st);
            }
            launch_nrm2(dt.as<double>(), n, dpart.as<double>(), nch, dnrm.as<double>() + 2, st);
            double tn2 = 0.0;
            PD_CK(cudaMemcpyAsync(&tn2, dnrm.as<double>() + 2, 8, cudaMemcpyDeviceToHost, st));
            PD_CK(cudaStreamSynchronize(st));
            if (std::sqrt(tn2) < 1e-14) break;
            double* vk = V + (size_t)k * n;
            double* avk = AV + (size_t)k * n;
            launch_scale(dt.as<double>(), dnrm.as<double>() + 2, n, vk, 1, st);
            mv(vk, avk);
            // new column k: G[i][k] = V_i . AV_k (i <= k); new row: G[k][i] = V_k . AV_i (i < k)
            launch_dots(V, n, k + 1, avk, n, dpart.as<double>(), nch, dd1.as<double>(), st);
            launch_dots(AV, n, k, vk, n, dpart.as<double>(), nch, dd2.as<double>(), st);
            k_place<<<1, 32, 0, st>>>(G, kmax, k, dd1.as<double>(), dd2.as<double>());
            PD_LAUNCHED();
            ++k;
        }
        // x = u / |u|
        launch_scale(du.as<double>(), dnrm.as<double>() + 1, n, x, 1, st);
    };
    run(max_iter);
    if (acc && refine_iters > 0) {
        PD_REQUIRE(acc->psi.size == n, DMRG_ERR_STATE, "refinement plan does not match the bond");
        cur = acc;
        run(refine_iters);
    }
    PD_CK(cudaStreamSynchronize(st));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return res;
}

}  // namespace pd
