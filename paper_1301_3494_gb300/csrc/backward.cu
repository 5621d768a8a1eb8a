// Backward of the projected-Hamiltonian matvec (the H_eff application of Sec. II), FP64.
//
// Forward: y[a',s1,s2,c'] = sum L[a',w,a] W1[w,s1,s1',w'] W2[w',s2,s2',w''] R[c',w'',c] x[a,s1',s2',c],
// in three stages over U(1) blocks:
//   X_w   = L_w x                                   (L stage, one block per MPO channel w)
//   Y_w'' = sum W12[w,s1,s1',s2,s2',w''] X_w        (MPO mix, W12 = sum_w' W1 W2)
//   y     = sum_w'' Y_w'' R_w''^T                   (R stage)
// Given ybar = dPhi/dy of a scalar Phi, reverse mode through the stages gives
//   Ybar_w'' = ybar R_w''              Rbar_w'' += ybar^T Y_w''
//   Xbar_w   = sum W12 Ybar_w''         W12bar    = <Ybar_w'', X_w> per two-site MPO entry
//   Lbar_w  += Xbar_w x^T               xbar      = sum_w L_w^T Xbar_w
//   W1bar[w,s1,s1',w'] = sum W12bar W2[w',s2,s2',w''],  W2bar[w',s2,s2',w''] = sum W12bar W1[w,s1,s1',w'].
// X and Y are recomputed from x here rather than kept from a forward call.  W12bar is formed for
// every entry W1 x W2 can produce (not only the nonzero entries of their product), so W1bar and
// W2bar are exact at every nonzero entry of W1 and W2; entries that are zero in W1 (resp. W2)
// get no gradient (the structure of the MPO is fixed).
#include <map>
#include <tuple>

#include "plans.h"

namespace pd {
Sec make_sec(int n, const int* q, const int* m);
SiteMPO make_site_mpo(int Dl, int Dr, int d, const int* fl, const int* fr, const double* W, const std::vector<int>& qn);
dmrg_status fail(const Error& e);
}  // namespace pd

using namespace pd;

namespace {

// dot of two equally shaped blocks: part[j] = sum_e a[a_off + e] b[b_off + e], e < len
struct DotJob {
    long long a_off, b_off, len;
};
__global__ void k_block_dot(const DotJob* __restrict__ jobs, const double* __restrict__ A, const double* __restrict__ B,
                            double* __restrict__ part) {
    const DotJob j = jobs[blockIdx.x];
    double s = 0.0;
    for (long long e = threadIdx.x; e < j.len; e += blockDim.x) s = fma(A[j.a_off + e], B[j.b_off + e], s);
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

// out[i] = sum_{t in [t0[i], t0[i+1])} coef[t] * in[idx[t]], in the listed order
__global__ void k_gather_sum(const int* __restrict__ t0, const int* __restrict__ idx, const double* __restrict__ coef,
                             const double* __restrict__ in, int n, double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int t = t0[i]; t < t0[i + 1]; ++t) s = fma(coef ? coef[t] : 1.0, in[idx[t]], s);
    out[i] = s;
}

std::vector<GTile> tiles64(const std::vector<GProb>& probs) {
    std::vector<GTile> t;
    for (int p = 0; p < (int)probs.size(); ++p)
        for (int m0 = 0; m0 < probs[p].M; m0 += 64)
            for (int n0 = 0; n0 < probs[p].N; n0 += 64) t.push_back({p, m0, n0, 0});
    return t;
}

// one grouped FP64 GEMM launch from host lists
void gemm64(const std::vector<GProb>& p, const std::vector<GSeg>& s, const double* A, const double* B, double* C,
            cudaStream_t st) {
    if (p.empty()) return;
    DBuf dp, ds, dt;
    const std::vector<GTile> t = tiles64(p);
    upload(dp, p, st);
    upload(ds, s, st);
    upload(dt, t, st);
    launch_gemm_simt<double>(dp.as<GProb>(), ds.as<GSeg>(), dt.as<GTile>(), (int)t.size(), A, B, C, st);
}

GProb prob(int M, int N, long long c_off, int sam, int sak, int sbn, int sbk, int scm, int scn, int seg0, int nseg,
           int accumulate) {
    GProb p{};
    p.M = M; p.N = N; p.seg0 = seg0; p.nseg = nseg; p.c_off = c_off;
    p.sam = sam; p.sak = sak; p.sbn = sbn; p.sbk = sbk; p.scm = scm; p.scn = scn;
    p.accumulate = accumulate; p.alpha = 1.0;
    return p;
}

}  // namespace

namespace pd {

void heff_backward(const Sec& bl, const Sec& br, const std::vector<int>& qn, const SiteMPO& w1, const SiteMPO& w2,
                   const double* L_dev, const double* R_dev, const double* x_dev, const double* ybar_dev,
                   double* xbar_dev, double* Lbar_dev, double* Rbar_dev, double* W1bar, double* W2bar,
                   cudaStream_t st) {
    {
        const TwoSiteMPO t = two_site_mpo(w1, w2);
        const PsiLayout P = psi_layout(bl, br, qn);
        const EnvLayout L = env_layout(bl, w1.fl, 0), R = env_layout(br, w2.fr, 0);
        const int d = (int)qn.size();
        const auto& pb = P.blk;
        const int nb = (int)pb.size();

        // X blocks for every channel w and psi block b with an L block
        struct XB { long long off; int rows, cols, iab, lb; };
        std::vector<XB> xb;
        std::vector<int> xidx((size_t)t.D0 * nb, -1);
        long long xsize = 0;
        for (int b = 0; b < nb; ++b)
            for (int w = 0; w < t.D0; ++w) {
                const int iab = bl.find(bl.q[pb[b].i] + t.f0[w]);
                if (iab < 0) continue;
                const int lb = L.at(iab, w);
                if (lb < 0) continue;
                xidx[(size_t)w * nb + b] = (int)xb.size();
                xb.push_back({xsize, bl.m[iab], pb[b].cols, iab, lb});
                xsize += (long long)bl.m[iab] * pb[b].cols;
            }
        // Ybar blocks for every output block o and channel w2 with an R block
        struct YB { long long off; int rows, cols, o, rb; };
        std::vector<YB> yb;
        std::vector<int> yidx((size_t)nb * t.D2, -1);
        long long ysize = 0;
        for (int o = 0; o < nb; ++o)
            for (int w2 = 0; w2 < t.D2; ++w2) {
                const int rb = R.at(pb[o].k, w2);
                if (rb < 0) continue;
                yidx[(size_t)o * t.D2 + w2] = (int)yb.size();
                yb.push_back({ysize, pb[o].rows, R.blk[rb].cols, o, rb});
                ysize += (long long)pb[o].rows * R.blk[rb].cols;
            }
        // mix terms from the nonzero two-site MPO entries: Y(o, w2) += v X(w, b)
        std::vector<std::vector<std::pair<int, double>>> yterm(yb.size()), xterm(xb.size());
        for (const auto& e : t.nz)
            for (int b = 0; b < nb; ++b) {
                if (pb[b].s1 != e.s1p || pb[b].s2 != e.s2p) continue;
                const int xi = xidx[(size_t)e.w * nb + b];
                if (xi < 0) continue;
                const int o = P.at(xb[xi].iab, e.s1, e.s2);
                if (o < 0) continue;
                const int yi = yidx[(size_t)o * t.D2 + e.w2];
                if (yi < 0) continue;
                PD_REQUIRE(yb[yi].cols == pb[b].cols, DMRG_ERR_QN, "MPO flux rule violated in the two-site operator");
                yterm[yi].push_back({xi, e.v});
                xterm[xi].push_back({yi, e.v});
            }

        DBuf dX, dY, dYb, dXb;
        dX.ensure(std::max<long long>(1, xsize) * 8, st);
        dY.ensure(std::max<long long>(1, ysize) * 8, st);
        dYb.ensure(std::max<long long>(1, ysize) * 8, st);
        dXb.ensure(std::max<long long>(1, xsize) * 8, st);
        PD_CK(cudaMemsetAsync(dY.p, 0, std::max<long long>(1, ysize) * 8, st));
        PD_CK(cudaMemsetAsync(dXb.p, 0, std::max<long long>(1, xsize) * 8, st));
        double* X = dX.as<double>();
        double* Y = dY.as<double>();
        double* Yb = dYb.as<double>();
        double* Xb = dXb.as<double>();

        // 1. X(w, b)[a'][c] = sum_a L[a'][a] x_b[a][c]
        {
            std::vector<GProb> p;
            std::vector<GSeg> s;
            for (int b = 0; b < nb; ++b)
                for (int w = 0; w < t.D0; ++w) {
                    const int xi = xidx[(size_t)w * nb + b];
                    if (xi < 0) continue;
                    const auto& B = pb[b];
                    // C(m = c, n = a') = sum_a A(m = c, k = a) B(n = a', k = a)
                    p.push_back(prob(B.cols, xb[xi].rows, xb[xi].off, 1, B.cols, B.rows, 1, 1, B.cols, (int)s.size(), 1, 0));
                    s.push_back({B.off, L.blk[xb[xi].lb].packed, B.rows, 0});
                }
            gemm64(p, s, x_dev, L_dev, X, st);
        }
        // 2. Y(o, w2) = sum v X(w, b)   (mixing jobs over the recomputed X)
        {
            std::vector<MixJob> mj;
            std::vector<MixTerm> mt;
            std::vector<long long> el;
            for (size_t y = 0; y < yb.size(); ++y) {
                if (yterm[y].empty()) continue;
                MixJob j{};
                j.dst = yb[y].off; j.rows = yb[y].rows; j.cols = yb[y].cols; j.ldo = yb[y].cols; j.zero_to = 0;
                j.t0 = (int)mt.size(); j.nt = (int)yterm[y].size();
                for (auto& tm : yterm[y]) mt.push_back({xb[tm.first].off, xb[tm.first].cols, 0, tm.second});
                mj.push_back(j);
                el.push_back((long long)j.rows * j.cols);
            }
            if (!mj.empty()) {
                DBuf dj, dt2, dc;
                const std::vector<int2> ch = make_chunks(el);
                upload(dj, mj, st);
                upload(dt2, mt, st);
                upload(dc, ch, st);
                launch_mix<double, double>(dj.as<MixJob>(), dc.as<int2>(), (int)ch.size(), dt2.as<MixTerm>(), X, Y, st);
            }
        }
        // 3. Ybar(o, w2)[a'][c] = sum_c' ybar_o[a'][c'] R[c'][c]
        {
            std::vector<GProb> p;
            std::vector<GSeg> s;
            for (size_t y = 0; y < yb.size(); ++y) {
                const auto& O = pb[yb[y].o];
                const auto& RB = R.blk[yb[y].rb];
                // C(m = c, n = a') = sum_c' A(m = c, k = c') B(n = a', k = c')
                p.push_back(prob(yb[y].cols, yb[y].rows, yb[y].off, 1, RB.cols, O.cols, 1, 1, yb[y].cols, (int)s.size(), 1, 0));
                s.push_back({RB.packed, O.off, O.cols, 0});
            }
            gemm64(p, s, R_dev, ybar_dev, Yb, st);
        }
        // 4. Rbar(k', w2)[c'][c] = sum over outputs o with k_o = k' of sum_a' ybar_o[a'][c'] Y(o, w2)[a'][c]
        {
            PD_CK(cudaMemsetAsync(Rbar_dev, 0, std::max<long long>(1, R.packed_size) * 8, st));
            std::vector<std::vector<int>> per_rb(R.blk.size());
            for (size_t y = 0; y < yb.size(); ++y)
                if (!yterm[y].empty()) per_rb[yb[y].rb].push_back((int)y);
            std::vector<GProb> p;
            std::vector<GSeg> s;
            for (size_t rb = 0; rb < R.blk.size(); ++rb) {
                if (per_rb[rb].empty()) continue;
                const auto& RB = R.blk[rb];
                const int seg0 = (int)s.size();
                for (int y : per_rb[rb]) s.push_back({yb[y].off, pb[yb[y].o].off, yb[y].rows, 0});
                // C(m = c, n = c') = sum_a' A(m = c, k = a') B(n = c', k = a')
                p.push_back(prob(RB.cols, RB.rows, RB.packed, 1, RB.cols, 1, RB.rows, 1, RB.cols, seg0,
                                 (int)per_rb[rb].size(), 0));
            }
            gemm64(p, s, Y, ybar_dev, Rbar_dev, st);
        }
        // 5. Xbar(w, b) = sum v Ybar(o, w2)   (transposed mix)
        {
            std::vector<MixJob> mj;
            std::vector<MixTerm> mt;
            std::vector<long long> el;
            for (size_t x = 0; x < xb.size(); ++x) {
                if (xterm[x].empty()) continue;
                MixJob j{};
                j.dst = xb[x].off; j.rows = xb[x].rows; j.cols = xb[x].cols; j.ldo = xb[x].cols; j.zero_to = 0;
                j.t0 = (int)mt.size(); j.nt = (int)xterm[x].size();
                for (auto& tm : xterm[x]) mt.push_back({yb[tm.first].off, yb[tm.first].cols, 0, tm.second});
                mj.push_back(j);
                el.push_back((long long)j.rows * j.cols);
            }
            if (!mj.empty()) {
                DBuf dj, dt2, dc;
                const std::vector<int2> ch = make_chunks(el);
                upload(dj, mj, st);
                upload(dt2, mt, st);
                upload(dc, ch, st);
                launch_mix<double, double>(dj.as<MixJob>(), dc.as<int2>(), (int)ch.size(), dt2.as<MixTerm>(), Yb, Xb, st);
            }
        }
        // 6. Lbar(iab, w)[a'][a] = sum_b sum_c Xbar(w, b)[a'][c] x_b[a][c]; the k-th contribution to
        //    each L block goes into launch k (accumulating for k > 0): strides differ per b
        {
            PD_CK(cudaMemsetAsync(Lbar_dev, 0, std::max<long long>(1, L.packed_size) * 8, st));
            std::vector<int> nth(L.blk.size(), 0);
            std::vector<std::vector<GProb>> p;
            std::vector<std::vector<GSeg>> s;
            for (int b = 0; b < nb; ++b)
                for (int w = 0; w < t.D0; ++w) {
                    const int xi = xidx[(size_t)w * nb + b];
                    if (xi < 0 || xterm[xi].empty()) continue;
                    const auto& B = pb[b];
                    const auto& LB = L.blk[xb[xi].lb];
                    const int k = nth[xb[xi].lb]++;
                    if ((int)p.size() <= k) { p.emplace_back(); s.emplace_back(); }
                    // C(m = a, n = a') = sum_c A(m = a, k = c) B(n = a', k = c)
                    p[k].push_back(prob(B.rows, LB.rows, LB.packed, B.cols, 1, B.cols, 1, 1, LB.cols, (int)s[k].size(), 1, 1));
                    s[k].push_back({B.off, xb[xi].off, B.cols, 0});
                }
            for (size_t k = 0; k < p.size(); ++k) gemm64(p[k], s[k], x_dev, Xb, Lbar_dev, st);
        }
        // 7. xbar_b[a][c] = sum_w sum_a' L(iab, w)[a'][a] Xbar(w, b)[a'][c]
        {
            PD_CK(cudaMemsetAsync(xbar_dev, 0, std::max<long long>(1, P.size) * 8, st));
            std::vector<GProb> p;
            std::vector<GSeg> s;
            for (int b = 0; b < nb; ++b) {
                const auto& B = pb[b];
                const int seg0 = (int)s.size();
                for (int w = 0; w < t.D0; ++w) {
                    const int xi = xidx[(size_t)w * nb + b];
                    if (xi < 0 || xterm[xi].empty()) continue;
                    s.push_back({xb[xi].off, L.blk[xb[xi].lb].packed, xb[xi].rows, 0});
                }
                if ((int)s.size() == seg0) continue;
                // C(m = c, n = a) = sum_a' A(m = c, k = a') B(n = a, k = a')
                p.push_back(prob(B.cols, B.rows, B.off, 1, B.cols, 1, B.rows, 1, B.cols, seg0, (int)s.size() - seg0, 0));
            }
            gemm64(p, s, Xb, L_dev, xbar_dev, st);
        }
        // 8. W12bar for every combination W1 x W2 produces, then W1bar / W2bar
        if (W1bar || W2bar) {
            struct Combo { int w, s1, s1p, s2, s2p, w2; };
            std::vector<Combo> combos;
            std::map<std::tuple<int, int, int, int, int, int>, int> cidx;
            // pairs (W1 entry, W2 entry, combo)
            struct Pair { long long i1, i2; int c; };
            std::vector<Pair> pairs;
            for (int w = 0; w < w1.Dl; ++w)
                for (int s1 = 0; s1 < d; ++s1)
                    for (int s1p = 0; s1p < d; ++s1p)
                        for (int wp = 0; wp < w1.Dr; ++wp) {
                            const long long i1 = (((long long)w * d + s1) * d + s1p) * w1.Dr + wp;
                            if (w1.W[i1] == 0.0) continue;
                            for (int s2 = 0; s2 < d; ++s2)
                                for (int s2p = 0; s2p < d; ++s2p)
                                    for (int w2i = 0; w2i < w2.Dr; ++w2i) {
                                        const long long i2 = (((long long)wp * d + s2) * d + s2p) * w2.Dr + w2i;
                                        if (w2.W[i2] == 0.0) continue;
                                        auto key = std::make_tuple(w, s1, s1p, s2, s2p, w2i);
                                        auto it = cidx.find(key);
                                        int c;
                                        if (it == cidx.end()) {
                                            c = (int)combos.size();
                                            cidx[key] = c;
                                            combos.push_back({w, s1, s1p, s2, s2p, w2i});
                                        } else c = it->second;
                                        pairs.push_back({i1, i2, c});
                                    }
                        }
            // dot jobs per combo (in combo order) over the psi blocks it connects
            std::vector<DotJob> jobs;
            std::vector<int> jt0(combos.size() + 1, 0), jidx;
            for (size_t c = 0; c < combos.size(); ++c) {
                jt0[c] = (int)jidx.size();
                const Combo& C = combos[c];
                for (int b = 0; b < nb; ++b) {
                    if (pb[b].s1 != C.s1p || pb[b].s2 != C.s2p) continue;
                    const int xi = xidx[(size_t)C.w * nb + b];
                    if (xi < 0) continue;
                    const int o = P.at(xb[xi].iab, C.s1, C.s2);
                    if (o < 0) continue;
                    const int yi = yidx[(size_t)o * t.D2 + C.w2];
                    if (yi < 0 || yb[yi].cols != pb[b].cols) continue;
                    jidx.push_back((int)jobs.size());
                    jobs.push_back({yb[yi].off, xb[xi].off, (long long)xb[xi].rows * xb[xi].cols});
                }
            }
            jt0[combos.size()] = (int)jidx.size();
            DBuf dj, dpart, djt0, djidx, dW12;
            upload(dj, jobs, st);
            dpart.ensure(std::max<size_t>(1, jobs.size()) * 8, st);
            upload(djt0, jt0, st);
            upload(djidx, jidx, st);
            dW12.ensure(std::max<size_t>(1, combos.size()) * 8, st);
            if (!jobs.empty()) {
                k_block_dot<<<(unsigned)jobs.size(), 256, 0, st>>>(dj.as<DotJob>(), Yb, X, dpart.as<double>());
                PD_LAUNCHED();
            }
            if (!combos.empty()) {
                k_gather_sum<<<((int)combos.size() + 127) / 128, 128, 0, st>>>(djt0.as<int>(), djidx.as<int>(), nullptr,
                                                                              dpart.as<double>(), (int)combos.size(),
                                                                              dW12.as<double>());
                PD_LAUNCHED();
            }
            // W1bar[i1] = sum over its pairs W12bar[c] W2[i2]; W2bar[i2] = sum W12bar[c] W1[i1]
            auto reduce = [&](bool first, double* out) {
                if (!out) return;
                const size_t nout = first ? w1.W.size() : w2.W.size();
                std::vector<std::vector<std::pair<int, double>>> lst(nout);
                for (const auto& pr : pairs)
                    if (first) lst[pr.i1].push_back({pr.c, w2.W[pr.i2]});
                    else lst[pr.i2].push_back({pr.c, w1.W[pr.i1]});
                std::vector<int> t0(nout + 1, 0), idx;
                std::vector<double> coef;
                for (size_t i = 0; i < nout; ++i) {
                    t0[i] = (int)idx.size();
                    for (auto& e : lst[i]) { idx.push_back(e.first); coef.push_back(e.second); }
                }
                t0[nout] = (int)idx.size();
                DBuf dt0, didx, dco, dout;
                upload(dt0, t0, st);
                upload(didx, idx, st);
                upload(dco, coef, st);
                dout.ensure(std::max<size_t>(1, nout) * 8, st);
                k_gather_sum<<<((int)nout + 127) / 128, 128, 0, st>>>(dt0.as<int>(), didx.as<int>(), dco.as<double>(),
                                                                     dW12.as<double>(), (int)nout, dout.as<double>());
                PD_LAUNCHED();
                PD_CK(cudaMemcpyAsync(out, dout.p, nout * 8, cudaMemcpyDeviceToHost, st));
                PD_CK(cudaStreamSynchronize(st));
            };
            reduce(true, W1bar);
            reduce(false, W2bar);
        }
        PD_CK(cudaStreamSynchronize(st));
    }
}

}  // namespace pd

extern "C" dmrg_status dmrg_heff_backward(const dmrg_bond_desc* bd, const double* L_dev, const double* R_dev,
                                          const double* x_dev, const double* ybar_dev, double* xbar_dev,
                                          double* Lbar_dev, double* Rbar_dev, double* W1bar, double* W2bar,
                                          void* stream) {
    try {
        PD_REQUIRE(bd && bd->d > 0 && bd->d <= 8 && bd->qn_local, DMRG_ERR_ARG, "bad bond descriptor");
        PD_REQUIRE(L_dev && R_dev && x_dev && ybar_dev && xbar_dev && Lbar_dev && Rbar_dev, DMRG_ERR_ARG,
                   "null buffer");
        std::vector<int> qn(bd->qn_local, bd->qn_local + bd->d);
        const Sec bl = make_sec(bd->nl, bd->ql, bd->ml), br = make_sec(bd->nr, bd->qr, bd->mr);
        const SiteMPO w1 = make_site_mpo(bd->D0, bd->D1, bd->d, bd->f0, bd->f1, bd->W1, qn);
        const SiteMPO w2 = make_site_mpo(bd->D1, bd->D2, bd->d, bd->f1, bd->f2, bd->W2, qn);
        heff_backward(bl, br, qn, w1, w2, L_dev, R_dev, x_dev, ybar_dev, xbar_dev, Lbar_dev, Rbar_dev, W1bar, W2bar,
                      (cudaStream_t)stream);
        return DMRG_OK;
    } catch (const Error& e) {
        return fail(e);
    }
}
