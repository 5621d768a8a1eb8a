// Householder QR of the charge-sector matrices of a two-site split, used to precondition the
// one-sided Jacobi SVD of Eq. (svd) (Sec. II) in the manner of Drmac and Veselic ("New fast and
// accurate Jacobi SVD algorithm", SIAM J. Matrix Anal. Appl. 29, 2008): W = Q R, then the
// one-sided Jacobi runs on the columns of X = R^T, whose rows are already graded by the QR, so it
// needs a few sweeps instead of the many it needs on W itself.  With X V_J = Y (orthogonal
// columns, Y = U_Y Sigma):
//   W = Q R = (Q V_J) Sigma U_Y^T,
// so the left singular vectors of W are Q V_J (orthonormal: a product of orthogonal factors), the
// singular values the column norms of Y, and the right singular vectors U_Y = Y Sigma^-1.
//
// The QR is blocked (LAPACK's geqrf / larft scheme, restated): panels of NB columns are factored
// by one CTA per sector in shared memory (one Householder reflector per column,
// H = I - tau v v^T, v(0) = 1), the panel's reflectors are accumulated into the compact form
// H_1 ... H_NB = I - V T V^T (T upper triangular), and the trailing columns are updated by the
// block reflector C <- C - V (T^T (V^T C)), many CTAs per sector.  Q is applied to the output
// the same way, panels in reverse order, with T in place of T^T.
#include <algorithm>
#include <vector>

#include "plans.h"

namespace pd {

namespace {

constexpr int QR_THREADS = 256;
constexpr int QR_TN = 32;        // columns of C per update CTA
constexpr int QR_CH = 64;        // rows per staged chunk in the update
constexpr int QR_SMEM_MAX = 226 * 1024;

template <class T> struct QrNB;
template <> struct QrNB<float> { static constexpr int v = 32; };
template <> struct QrNB<double> { static constexpr int v = 16; };

// One panel of every active sector: rows c0..p-1, columns c0..c0+nb-1 of W (column-major, ld p).
// Factors it in place (R on and above the diagonal, reflector entries v(1..) below it) and
// writes the panel's T (NB x NB, column-major) to Tf.
template <class T, int NB>
__global__ void __launch_bounds__(QR_THREADS) k_qr_panel(const QrSec* __restrict__ secs, const int* __restrict__ act,
                                                         int c0, T* __restrict__ W, T* __restrict__ Tf) {
    extern __shared__ __align__(16) unsigned char qr_smem[];
    constexpr int LDP = NB + 1;
    constexpr int NW = QR_THREADS / 32;
    const QrSec s = secs[act[blockIdx.x]];
    const int nb = min(NB, s.n - c0);
    const int rows = s.p - c0;
    T* P = reinterpret_cast<T*>(qr_smem);                 // rows x LDP, row-major
    T* red = P + (size_t)rows * LDP;                      // NW x (NB + 1) partial sums
    T* wv = red + NW * (NB + 1);                          // NB: v^T a of the current column
    T* tau = wv + NB;                                     // NB
    T* G = tau + NB;                                      // NB x NB: V^T V (upper part)
    T* Ts = G + NB * NB;                                  // NB x NB: the panel's T
    T* scal = Ts + NB * NB;                               // beta, inv
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    T* Wp = W + s.w_off + (long long)c0 * s.p + c0;       // panel origin
    for (int j = 0; j < nb; ++j)
        for (int r = tid; r < rows; r += QR_THREADS) P[r * LDP + j] = Wp[(long long)j * s.p + r];
    for (int j = nb; j < NB; ++j)
        for (int r = tid; r < rows; r += QR_THREADS) P[r * LDP + j] = T(0);
    __syncthreads();
    for (int j = 0; j < nb; ++j) {
        // sig2 = sum_{r > j} x_r^2, d[jj] = sum_{r > j} x_r a_{r, jj} for jj > j
        T acc[NB + 1];
#pragma unroll
        for (int q = 0; q <= NB; ++q) acc[q] = T(0);
        for (int r = j + 1 + tid; r < rows; r += QR_THREADS) {
            const T x = P[r * LDP + j];
            acc[0] += x * x;
#pragma unroll
            for (int jj = 0; jj < NB; ++jj) acc[jj + 1] += (jj > j) ? x * P[r * LDP + jj] : T(0);
        }
#pragma unroll
        for (int q = 0; q <= NB; ++q) {
            T v = acc[q];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) red[wid * (NB + 1) + q] = v;
        }
        __syncthreads();
        if (tid <= NB) {
            T v = T(0);
#pragma unroll
            for (int w = 0; w < NW; ++w) v += red[w * (NB + 1) + tid];
            red[tid] = v;                      // warp 0's row holds the totals (read after the sync)
        }
        __syncthreads();
        if (tid == 0) {
            const T alpha = P[j * LDP + j], sig2 = red[0];
            T beta = alpha, tj = T(0), inv = T(0);
            if (sig2 > T(0)) {
                const T nrm = sqrt(alpha * alpha + sig2);
                beta = alpha >= T(0) ? -nrm : nrm;
                tj = (beta - alpha) / beta;
                inv = T(1) / (alpha - beta);
            }
            tau[j] = tj;
            scal[0] = beta;
            scal[1] = inv;
        }
        __syncthreads();
        const T tj = tau[j], inv = scal[1];
        // w_jj = v^T a_jj = a_{j, jj} + inv d[jj]
        if (tid < NB) wv[tid] = (tid > j && tid < nb) ? P[j * LDP + tid] + inv * red[tid + 1] : T(0);
        __syncthreads();
        for (int r = j + tid; r < rows; r += QR_THREADS) {
            const T vr = (r == j) ? T(1) : inv * P[r * LDP + j];
            const T f = tj * vr;
#pragma unroll
            for (int jj = 0; jj < NB; ++jj)
                if (jj > j) P[r * LDP + jj] -= f * wv[jj];
            P[r * LDP + j] = (r == j) ? scal[0] : vr;
        }
        __syncthreads();
    }
    // G = V^T V over the panel's reflectors (i < j): v_i(j) + sum_{r > j} v_i(r) v_j(r)
    for (int e = tid; e < NB * NB; e += QR_THREADS) {
        const int i = e % NB, j = e / NB;
        T g = T(0);
        if (i < j && j < nb) {
            g = P[j * LDP + i];
            for (int r = j + 1; r < rows; ++r) g += P[r * LDP + i] * P[r * LDP + j];
        }
        G[i + j * NB] = g;
    }
    __syncthreads();
    // T: T(j, j) = tau_j, T(0:j, j) = -tau_j T(0:j, 0:j) G(0:j, j)  (one warp, column by column)
    if (wid == 0) {
        for (int j = 0; j < NB; ++j) {
            T y = T(0);
            if (lane < j && j < nb)
                for (int k = lane; k < j; ++k) y += Ts[lane + k * NB] * G[k + j * NB];
            __syncwarp();
            if (lane < NB) Ts[lane + j * NB] = (j < nb) ? (lane < j ? -tau[j] * y : (lane == j ? tau[j] : T(0))) : T(0);
            __syncwarp();
        }
    }
    __syncthreads();
    T* Tp = Tf + s.t_off + (long long)(c0 / NB) * NB * NB;
    for (int e = tid; e < NB * NB; e += QR_THREADS) Tp[e] = Ts[e];
    for (int j = 0; j < nb; ++j)
        for (int r = tid; r < rows; r += QR_THREADS) Wp[(long long)j * s.p + r] = P[r * LDP + j];
}

// One tile of QR_TN columns of C (column-major, ld p, rows c0..p-1 of sector tile.x starting at
// column tile.y): C <- C - V (op(T) (V^T C)) with the reflectors of panel c0 / NB of W, op(T) = T^T
// (trans = 1, applying Q^T) or T (trans = 0, applying Q).
template <class T, int NB>
__global__ void __launch_bounds__(QR_THREADS) k_qr_apply(const QrSec* __restrict__ secs, const int2* __restrict__ tiles,
                                                         int c0, int trans, const T* W, const T* __restrict__ Tf,
                                                         T* Cbuf) {
    __shared__ T Vs[QR_CH][NB + 1];
    __shared__ T Cs[QR_CH][QR_TN + 1];
    __shared__ T Z[NB][QR_TN + 1];
    __shared__ T Z2[NB][QR_TN + 1];
    __shared__ T Ts[NB][NB + 1];
    const int2 tl = tiles[blockIdx.x];
    const QrSec s = secs[tl.x];
    const int col0 = tl.y;
    const int nc = min(QR_TN, s.n - col0);
    const int nb = min(NB, s.n - c0);
    const int rows = s.p - c0;
    const int tid = threadIdx.x;
    const T* V = W + s.w_off + (long long)c0 * s.p + c0;           // V(r, i) = V[i * p + r]
    T* C = Cbuf + s.w_off + (long long)col0 * s.p + c0;            // C(r, j) = C[j * p + r]
    const T* Tp = Tf + s.t_off + (long long)(c0 / NB) * NB * NB;
    for (int e = tid; e < NB * NB; e += QR_THREADS) {
        const int i = e % NB, j = e / NB;
        const T t = Tp[i + j * NB];
        if (trans) Ts[j][i] = t; else Ts[i][j] = t;   // Ts = op(T)
    }
    // Z = V^T C: thread -> Z(zi, zj0..zj0+ZPT-1)
    constexpr int ZPT = NB * QR_TN / QR_THREADS;     // 4 (NB = 32) or 2 (NB = 16)
    const int zi = tid / (QR_TN / ZPT), zj0 = (tid % (QR_TN / ZPT)) * ZPT;
    T za[ZPT];
#pragma unroll
    for (int q = 0; q < ZPT; ++q) za[q] = T(0);
    auto stage_v = [&](int r0, int len) {
        for (int e = tid; e < QR_CH * NB; e += QR_THREADS) {
            const int r = e % QR_CH, i = e / QR_CH;
            const int rr = r0 + r;
            T v = T(0);
            if (r < len && i < nb) v = rr > i ? V[(long long)i * s.p + rr] : (rr == i ? T(1) : T(0));
            Vs[r][i] = v;
        }
    };
    for (int r0 = 0; r0 < rows; r0 += QR_CH) {
        const int len = min(QR_CH, rows - r0);
        stage_v(r0, len);
        for (int e = tid; e < QR_CH * QR_TN; e += QR_THREADS) {
            const int r = e % QR_CH, j = e / QR_CH;
            Cs[r][j] = (r < len && j < nc) ? C[(long long)j * s.p + r0 + r] : T(0);
        }
        __syncthreads();
        for (int r = 0; r < len; ++r) {
            const T v = Vs[r][zi];
#pragma unroll
            for (int q = 0; q < ZPT; ++q) za[q] += v * Cs[r][zj0 + q];
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < ZPT; ++q) Z[zi][zj0 + q] = za[q];
    __syncthreads();
    // Z2 = op(T) Z
    for (int e = tid; e < NB * QR_TN; e += QR_THREADS) {
        const int i = e / QR_TN, j = e % QR_TN;
        T a = T(0);
#pragma unroll 4
        for (int k = 0; k < NB; ++k) a += Ts[i][k] * Z[k][j];
        Z2[i][j] = a;
    }
    __syncthreads();
    // C -= V Z2: thread -> row r of the chunk, columns cq..cq+CPT-1
    constexpr int RPT = QR_THREADS / QR_CH;            // 4 column groups
    constexpr int CPT = QR_TN / RPT;                   // 8 columns each
    const int rr_ = tid % QR_CH, cq = (tid / QR_CH) * CPT;
    for (int r0 = 0; r0 < rows; r0 += QR_CH) {
        const int len = min(QR_CH, rows - r0);
        stage_v(r0, len);
        __syncthreads();
        if (rr_ < len) {
            T o[CPT];
#pragma unroll
            for (int q = 0; q < CPT; ++q) o[q] = T(0);
#pragma unroll 4
            for (int i = 0; i < NB; ++i) {
                const T v = Vs[rr_][i];
#pragma unroll
                for (int q = 0; q < CPT; ++q) o[q] += v * Z2[i][cq + q];
            }
#pragma unroll
            for (int q = 0; q < CPT; ++q)
                if (cq + q < nc) C[(long long)(cq + q) * s.p + r0 + rr_] -= o[q];
        }
        __syncthreads();
    }
}

// X = R^T (n x n, column-major at x_off): X(i, j) = R(j, i) = W(j, i) for j <= i, else 0.
template <class T>
__global__ void k_qr_rt(const QrSec* __restrict__ secs, const long long* __restrict__ x_off, const T* __restrict__ W,
                        T* __restrict__ X) {
    const QrSec s = secs[blockIdx.y];
    const long long nn = (long long)s.n * s.n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nn; e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % s.n), j = (int)(e / s.n);
        X[x_off[blockIdx.y] + e] = (j <= i) ? W[s.w_off + j + (long long)i * s.p] : T(0);
    }
}

// Per sector column j (one CTA): sigma = |Y(:, j)|; Y(:, j) <- Y(:, j) / sigma (0 if sigma = 0);
// Wout(0:n, j) = V_J(:, j) sigma, Wout(n:p, j) = 0.
template <class T>
__global__ void k_qr_post(const QrSec* __restrict__ secs, const int2* __restrict__ cols, const long long* __restrict__ x_off,
                          T* __restrict__ Y, const T* __restrict__ VJ, T* __restrict__ Wout) {
    __shared__ double part[32];
    const int2 c = cols[blockIdx.x];
    const QrSec s = secs[c.x];
    const int j = c.y;
    T* y = Y + x_off[c.x] + (long long)j * s.n;
    double a = 0.0;
    for (int r = threadIdx.x; r < s.n; r += blockDim.x) a += (double)y[r] * (double)y[r];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
        part[0] = sqrt(t);
    }
    __syncthreads();
    const double sig = part[0];
    const T inv = sig > 0.0 ? T(1.0 / sig) : T(0);
    const T* v = VJ + x_off[c.x] + (long long)j * s.n;
    T* w = Wout + s.w_off + (long long)j * s.p;
    for (int r = threadIdx.x; r < s.n; r += blockDim.x) {
        y[r] *= inv;
        w[r] = v[r] * T(sig);
    }
    for (int r = s.n + threadIdx.x; r < s.p; r += blockDim.x) w[r] = T(0);
}

}  // namespace

int qr_max_rows(bool f64) {
    const size_t es = f64 ? 8 : 4;
    const int nb = f64 ? QrNB<double>::v : QrNB<float>::v;
    const size_t fixed = es * ((size_t)(QR_THREADS / 32) * (nb + 1) + 2 * nb + 2 * (size_t)nb * nb + 2) + 64;
    return (int)((QR_SMEM_MAX - fixed) / (es * (nb + 1)));
}

template <class T>
void QrPlan::build(const std::vector<SvdSec>& ss, cudaStream_t st) {
    constexpr int NB = QrNB<T>::v;
    secs.clear();
    long long toff = 0;
    int maxn = 0;
    max_rows = 0;
    for (const auto& x : ss) {
        QrSec q{};
        q.w_off = x.w_off;
        q.t_off = toff;
        q.p = x.p;
        q.n = x.n;
        toff += (long long)((x.n + NB - 1) / NB) * NB * NB;
        maxn = std::max(maxn, x.n);
        max_rows = std::max(max_rows, x.p);
        secs.push_back(q);
    }
    ok = !secs.empty() && max_rows <= qr_max_rows(sizeof(T) == 8);
    if (!ok) return;
    npanel = (maxn + NB - 1) / NB;
    std::vector<int> act;
    std::vector<int2> trail, all;
    act_off.assign(npanel + 1, 0);
    trail_off.assign(npanel + 1, 0);
    for (int k = 0; k < npanel; ++k) {
        const int c0 = k * NB;
        act_off[k] = (int)act.size();
        trail_off[k] = (int)trail.size();
        for (int s = 0; s < (int)secs.size(); ++s) {
            if (secs[s].n <= c0) continue;
            act.push_back(s);
            for (int c = c0 + NB; c < secs[s].n; c += QR_TN) trail.push_back(make_int2(s, c));
        }
    }
    act_off[npanel] = (int)act.size();
    trail_off[npanel] = (int)trail.size();
    // tiles over all columns of the sectors that have panel k, per panel
    all_off.assign(npanel + 1, 0);
    for (int k = 0; k < npanel; ++k) {
        all_off[k] = (int)all.size();
        for (int s = 0; s < (int)secs.size(); ++s) {
            if (secs[s].n <= k * NB) continue;
            for (int c = 0; c < secs[s].n; c += QR_TN) all.push_back(make_int2(s, c));
        }
    }
    all_off[npanel] = (int)all.size();
    std::vector<int2> cols;
    std::vector<long long> xo;
    for (int s = 0; s < (int)secs.size(); ++s) {
        for (int j = 0; j < secs[s].n; ++j) cols.push_back(make_int2(s, j));
        xo.push_back(ss[s].v_off);
    }
    ncols = (int)cols.size();
    upload(dsecs, secs, st);
    upload(dact, act, st);
    upload(dtrail, trail, st);
    upload(dall, all, st);
    upload(dcols, cols, st);
    upload(dxoff, xo, st);
    dT.ensure((size_t)std::max<long long>(1, toff) * sizeof(T), st);
}

template <class T>
void QrPlan::factor(T* W, cudaStream_t st) {
    constexpr int NB = QrNB<T>::v;
    static const cudaError_t attr =
        cudaFuncSetAttribute(k_qr_panel<T, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, QR_SMEM_MAX);
    PD_CK(attr);
    const size_t smem = sizeof(T) * ((size_t)max_rows * (NB + 1) + (size_t)(QR_THREADS / 32) * (NB + 1) + 2 * NB +
                                     2 * (size_t)NB * NB + 2);
    for (int k = 0; k < npanel; ++k) {
        const int na = act_off[k + 1] - act_off[k];
        if (na == 0) continue;
        k_qr_panel<T, NB><<<na, QR_THREADS, smem, st>>>(dsecs.as<QrSec>(), dact.as<int>() + act_off[k], k * NB, W,
                                                        dT.as<T>());
        PD_LAUNCHED();
        const int nt = trail_off[k + 1] - trail_off[k];
        if (nt == 0) continue;
        k_qr_apply<T, NB><<<nt, QR_THREADS, 0, st>>>(dsecs.as<QrSec>(), dtrail.as<int2>() + trail_off[k], k * NB, 1, W,
                                                     dT.as<T>(), W);
        PD_LAUNCHED();
    }
}

template <class T>
void QrPlan::form_rt(const T* W, T* X, cudaStream_t st) {
    dim3 g(64, (unsigned)secs.size());
    k_qr_rt<T><<<g, 256, 0, st>>>(dsecs.as<QrSec>(), dxoff.as<long long>(), W, X);
    PD_LAUNCHED();
}

template <class T>
void QrPlan::finish(const T* W, T* Y, const T* VJ, T* Wout, cudaStream_t st) {
    constexpr int NB = QrNB<T>::v;
    if (ncols > 0) {
        k_qr_post<T><<<ncols, 128, 0, st>>>(dsecs.as<QrSec>(), dcols.as<int2>(), dxoff.as<long long>(), Y, VJ, Wout);
        PD_LAUNCHED();
    }
    for (int k = npanel - 1; k >= 0; --k) {
        const int nt = all_off[k + 1] - all_off[k];
        if (nt == 0) continue;
        k_qr_apply<T, NB><<<nt, QR_THREADS, 0, st>>>(dsecs.as<QrSec>(), dall.as<int2>() + all_off[k], k * NB, 0, W,
                                                     dT.as<T>(), Wout);
        PD_LAUNCHED();
    }
}

template void QrPlan::build<float>(const std::vector<SvdSec>&, cudaStream_t);
template void QrPlan::build<double>(const std::vector<SvdSec>&, cudaStream_t);
template void QrPlan::factor<float>(float*, cudaStream_t);
template void QrPlan::factor<double>(double*, cudaStream_t);
template void QrPlan::form_rt<float>(const float*, float*, cudaStream_t);
template void QrPlan::form_rt<double>(const double*, double*, cudaStream_t);
template void QrPlan::finish<float>(const float*, float*, const float*, float*, cudaStream_t);
template void QrPlan::finish<double>(const double*, double*, const double*, double*, cudaStream_t);

}  // namespace pd
