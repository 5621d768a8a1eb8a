// FP64 projected-Hamiltonian matvec that allocates no device memory.
//
// For callers that cannot call cudaMalloc -- e.g. code running under an external memory
// manager that owns every device allocation, or a host thread that must not touch the CUDA
// allocator -- this entry point takes the same inputs and outputs as dmrg_heff_apply in FP64
// and keeps all of its scratch (job lists, the L-stage intermediate X and the MPO-mixed Y) in
// one file-scope device array of fixed size.  Operands are read directly in the packed block
// layout, so no operand copies are made.
//
// Set-up: the first call on a device (with that device current) resolves the array's device
// address with cudaGetSymbolAddress and caches it for that device; make that first call before
// any stream capture.  Every call shares the array and leaves its contents behind: the
// kernels overwrite everything they read, and the output vector is cleared by the call.
// Calls whose GPU work overlaps (different streams, or different host threads without
// ordering) race on the array.
#include <mutex>

#include "plans.h"

namespace pd {
Sec make_sec(int n, const int* q, const int* m);
SiteMPO make_site_mpo(int Dl, int Dr, int d, const int* fl, const int* fr, const double* W, const std::vector<int>& qn);
extern thread_local std::string g_last_error;
}  // namespace pd

using namespace pd;

namespace {

constexpr size_t kScratchBytes = size_t(64) << 20;          // 64 MiB, resident on every GPU that loads the library
__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_ptr[64] = {};

void* scratch_for_current_device() {
    int dev = 0;
    PD_CK(cudaGetDevice(&dev));
    PD_REQUIRE(dev >= 0 && dev < 64, DMRG_ERR_CAPACITY, "device ordinal beyond 63");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        PD_REQUIRE(e == cudaSuccess && p != nullptr, DMRG_ERR_CUDA,
                   std::string("cudaGetSymbolAddress of the scratch array failed: ") + cudaGetErrorString(e));
        g_scratch_ptr[dev] = p;
    }
    return g_scratch_ptr[dev];
}

// Bump placement inside the scratch array (host-side offsets, 256-byte aligned).
struct Arena {
    char* base;
    size_t used = 0;
    template <class T>
    T* take(size_t count) {
        size_t off = (used + 255) & ~size_t(255);
        size_t bytes = std::max<size_t>(1, count) * sizeof(T);
        PD_REQUIRE(off + bytes <= kScratchBytes, DMRG_ERR_CAPACITY,
                   "problem too large for the 64 MiB scratch of dmrg_heff_apply_noalloc");
        used = off + bytes;
        return reinterpret_cast<T*>(base + off);
    }
};

template <class T>
void put(T* dev, const std::vector<T>& h, cudaStream_t st) {
    if (!h.empty()) PD_CK(cudaMemcpyAsync(dev, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, st));
}

std::vector<GTile> tiles_of(const std::vector<GProb>& probs) {
    std::vector<GTile> t;
    for (int p = 0; p < (int)probs.size(); ++p)
        for (int m0 = 0; m0 < probs[p].M; m0 += 64)
            for (int n0 = 0; n0 < probs[p].N; n0 += 64) t.push_back({p, m0, n0, 0});
    return t;
}

}  // namespace

extern "C" dmrg_status dmrg_heff_apply_noalloc(const dmrg_bond_desc* bd, const double* L_dev, const double* R_dev,
                                               const double* x_dev, double* y_dev, void* stream) {
    try {
        PD_REQUIRE(bd && bd->d > 0 && bd->d <= 8 && bd->qn_local, DMRG_ERR_ARG, "bad bond descriptor");
        PD_REQUIRE(L_dev && R_dev && x_dev && y_dev, DMRG_ERR_ARG, "null buffer");
        cudaStream_t st = (cudaStream_t)stream;
        std::vector<int> qn(bd->qn_local, bd->qn_local + bd->d);
        const Sec bl = make_sec(bd->nl, bd->ql, bd->ml), br = make_sec(bd->nr, bd->qr, bd->mr);
        const SiteMPO w1 = make_site_mpo(bd->D0, bd->D1, bd->d, bd->f0, bd->f1, bd->W1, qn);
        const SiteMPO w2 = make_site_mpo(bd->D1, bd->D2, bd->d, bd->f1, bd->f2, bd->W2, qn);
        const TwoSiteMPO t = two_site_mpo(w1, w2);
        const PsiLayout P = psi_layout(bl, br, qn);
        const EnvLayout L = env_layout(bl, w1.fl, 0), R = env_layout(br, w2.fr, 0);
        const int d = (int)qn.size();
        const auto& pb = P.blk;

        // L stage, operands in packed layout: X[w,b][a'][c] = sum_a L_w[a'][a] psi_b[a][c]
        std::vector<char> used((size_t)t.D0 * d * d, 0);
        for (const auto& e : t.nz) used[((size_t)e.w * d + e.s1p) * d + e.s2p] = 1;
        struct XB { long long off; int rows, cols, iab; };
        std::vector<XB> xblk;
        std::vector<int> xindex((size_t)t.D0 * pb.size(), -1);
        std::vector<GProb> lp;
        std::vector<GSeg> ls;
        long long xsize = 0;
        for (int b = 0; b < (int)pb.size(); ++b) {
            const auto& B = pb[b];
            for (int w = 0; w < t.D0; ++w) {
                if (!used[((size_t)w * d + B.s1) * d + B.s2]) continue;
                int iab = bl.find(bl.q[B.i] + t.f0[w]);
                if (iab < 0) continue;
                int lb = L.at(iab, w);
                if (lb < 0) continue;
                xindex[(size_t)w * pb.size() + b] = (int)xblk.size();
                xblk.push_back({xsize, bl.m[iab], B.cols, iab});
                GProb p{};
                p.M = B.cols; p.N = bl.m[iab]; p.seg0 = (int)ls.size(); p.nseg = 1; p.c_off = xsize;
                p.sam = 1; p.sak = B.cols; p.sbn = B.rows; p.sbk = 1; p.scm = 1; p.scn = B.cols; p.alpha = 1.0;
                ls.push_back({B.off, L.blk[lb].packed, B.rows, 0});
                lp.push_back(p);
                xsize += (long long)bl.m[iab] * B.cols;
            }
        }
        // MPO mix into Y (packed [a'][c]) and the R-stage segments per output block
        std::vector<std::vector<std::pair<int, double>>> yterms;   // per Y block: (X block, coef)
        std::vector<int> ykey_o, ykey_w2;
        std::vector<std::vector<int>> out_y(pb.size());           // Y blocks feeding each output
        {
            std::vector<int> ymap((size_t)pb.size() * t.D2, -1);
            for (const auto& e : t.nz)
                for (int b = 0; b < (int)pb.size(); ++b) {
                    const auto& B = pb[b];
                    if (B.s1 != e.s1p || B.s2 != e.s2p) continue;
                    int xi = xindex[(size_t)e.w * pb.size() + b];
                    if (xi < 0) continue;
                    int o = P.at(xblk[xi].iab, e.s1, e.s2);
                    if (o < 0 || R.at(pb[o].k, e.w2) < 0) continue;
                    int& yi = ymap[(size_t)o * t.D2 + e.w2];
                    if (yi < 0) {
                        yi = (int)yterms.size();
                        yterms.emplace_back();
                        ykey_o.push_back(o);
                        ykey_w2.push_back(e.w2);
                        out_y[o].push_back(yi);
                    }
                    yterms[yi].push_back({xi, e.v});
                }
        }
        std::vector<MixJob> mj;
        std::vector<MixTerm> mt;
        std::vector<long long> yoff(yterms.size());
        std::vector<long long> melems;
        long long ysize = 0;
        for (size_t y = 0; y < yterms.size(); ++y) {
            const XB& x0 = xblk[yterms[y].front().first];
            yoff[y] = ysize;
            MixJob j{};
            j.dst = ysize; j.rows = x0.rows; j.cols = x0.cols; j.ldo = x0.cols; j.zero_to = 0;
            j.t0 = (int)mt.size(); j.nt = (int)yterms[y].size();
            for (auto& tm : yterms[y]) mt.push_back({xblk[tm.first].off, xblk[tm.first].cols, 0, tm.second});
            mj.push_back(j);
            melems.push_back((long long)j.rows * j.cols);
            ysize += (long long)x0.rows * x0.cols;
        }
        const std::vector<int2> mchunks = make_chunks(melems);
        // R stage: out[a'][c'] += sum_c Y[a'][c] R_w''[c'][c]; the k-th feeding Y block of every
        // output goes into launch k (accumulating for k > 0), so no launch writes a block twice
        size_t nlaunch = 0;
        for (auto& v : out_y) nlaunch = std::max(nlaunch, v.size());
        std::vector<std::vector<GProb>> rp(nlaunch);
        std::vector<std::vector<GSeg>> rs(nlaunch);
        for (int o = 0; o < (int)pb.size(); ++o)
            for (size_t k = 0; k < out_y[o].size(); ++k) {
                int y = out_y[o][k];
                const auto& O = pb[o];
                int rb = R.at(O.k, ykey_w2[y]);
                int mc = R.blk[rb].cols;
                GProb p{};
                p.M = O.cols; p.N = O.rows; p.seg0 = (int)rs[k].size(); p.nseg = 1; p.c_off = O.off;
                p.sam = mc; p.sak = 1; p.sbn = mc; p.sbk = 1; p.scm = 1; p.scn = O.cols;
                p.accumulate = k > 0 ? 1 : 0; p.alpha = 1.0;
                rs[k].push_back({R.blk[rb].packed, yoff[y], mc, 0});
                rp[k].push_back(p);
            }

        // place everything in the scratch array
        Arena ar{static_cast<char*>(scratch_for_current_device())};
        double* X = ar.take<double>(xsize);
        double* Y = ar.take<double>(ysize);
        const std::vector<GTile> lt = tiles_of(lp);
        GProb* d_lp = ar.take<GProb>(lp.size());
        GSeg* d_ls = ar.take<GSeg>(ls.size());
        GTile* d_lt = ar.take<GTile>(lt.size());
        MixJob* d_mj = ar.take<MixJob>(mj.size());
        MixTerm* d_mt = ar.take<MixTerm>(mt.size());
        int2* d_mc = ar.take<int2>(mchunks.size());
        std::vector<GProb*> d_rp(nlaunch);
        std::vector<GSeg*> d_rs(nlaunch);
        std::vector<GTile*> d_rt(nlaunch);
        std::vector<std::vector<GTile>> rt(nlaunch);
        for (size_t k = 0; k < nlaunch; ++k) {
            rt[k] = tiles_of(rp[k]);
            d_rp[k] = ar.take<GProb>(rp[k].size());
            d_rs[k] = ar.take<GSeg>(rs[k].size());
            d_rt[k] = ar.take<GTile>(rt[k].size());
        }
        put(d_lp, lp, st);
        put(d_ls, ls, st);
        put(d_lt, lt, st);
        put(d_mj, mj, st);
        put(d_mt, mt, st);
        put(d_mc, mchunks, st);
        for (size_t k = 0; k < nlaunch; ++k) {
            put(d_rp[k], rp[k], st);
            put(d_rs[k], rs[k], st);
            put(d_rt[k], rt[k], st);
        }
        PD_CK(cudaMemsetAsync(y_dev, 0, sizeof(double) * std::max<long long>(1, P.size), st));
        launch_gemm_simt<double>(d_lp, d_ls, d_lt, (int)lt.size(), x_dev, L_dev, X, st);
        launch_mix<double, double>(d_mj, d_mc, (int)mchunks.size(), d_mt, X, Y, st);
        for (size_t k = 0; k < nlaunch; ++k)
            launch_gemm_simt<double>(d_rp[k], d_rs[k], d_rt[k], (int)rt[k].size(), R_dev, Y, y_dev, st);
        // the host-side lists above are pageable, so every copy was staged before returning
        return DMRG_OK;
    } catch (const Error& e) {
        g_last_error = e.msg;
        return e.st;
    }
}
