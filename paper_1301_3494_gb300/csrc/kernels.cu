// FP64 / memory-bound kernels of the two-site DMRG step.
//
//  * k_gemm64       grouped, strided FP64 GEMM (the parity-mode contractions of the projected
//                   Hamiltonian and of the projected-operator updates, Sec. II)
//  * k_copy/k_mix   block gathers, transposes, MPO channel mixing (memory-bound)
//  * k_diag         diagonal of the projected Hamiltonian (Davidson preconditioner)
//  * Davidson       dot products, Ritz vectors, residuals, Gram-Schmidt, small Jacobi eigensolver
//  * SVD            batched one-sided (Hestenes) Jacobi SVD per charge sector, Eq. (svd)
//  * truncation     global keep-largest-m selection over all sectors (single CTA)
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <type_traits>
#include <vector>

#include "grid_sync.cuh"
#include "internal.h"


namespace pd {

namespace {

template <class T>
__device__ __forceinline__ double to_d(T x) { return (double)x; }
template <>
__device__ __forceinline__ double to_d<__nv_bfloat16>(__nv_bfloat16 x) { return (double)__bfloat162float(x); }

template <class T>
__device__ __forceinline__ T from_d(double x) { return (T)x; }
template <>
__device__ __forceinline__ __nv_bfloat16 from_d<__nv_bfloat16>(double x) { return __float2bfloat16_rn((float)x); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum (blockDim.x multiple of 32, <= 1024); result valid in every thread.
__device__ double block_sum(double v) {
    __shared__ double red[32];
    __shared__ double total;
    v = warp_sum(v);
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    if (wid == 0) {
        int nw = blockDim.x >> 5;
        double x = lane < nw ? red[lane] : 0.0;
        x = warp_sum(x);
        if (lane == 0) total = x;
    }
    __syncthreads();
    return total;
}

// ------------------------------------------------------------------------------------------
// Grouped SIMT GEMM (FP64 or FP32): 64x64 output tile per CTA, 256 threads, 4x4 per thread,
// K chunks of 16.
// ------------------------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(256) k_gemm_simt(const GProb* __restrict__ probs,
                                                   const GSeg* __restrict__ segs,
                                                   const GTile* __restrict__ tiles,
                                                   const T* __restrict__ A,
                                                   const T* __restrict__ B,
                                                   T* __restrict__ C) {
    __shared__ T As[16][65];
    __shared__ T Bs[16][65];
    const GTile t = tiles[blockIdx.x];
    const GProb p = probs[t.prob];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
    for (int sgi = 0; sgi < p.nseg; ++sgi) {
        const GSeg sg = segs[p.seg0 + sgi];
        for (int k0 = 0; k0 < sg.K; k0 += 16) {
            for (int e = tid; e < 1024; e += 256) {
                int kk = e & 15, mm = e >> 4;
                int m = t.m0 + mm, k = k0 + kk;
                T va = T(0), vb = T(0);
                if (m < p.M && k < sg.K) va = A[sg.a_off + (long long)m * p.sam + (long long)k * p.sak];
                int n = t.n0 + mm;
                if (n < p.N && k < sg.K) vb = B[sg.b_off + (long long)n * p.sbn + (long long)k * p.sbk];
                As[kk][mm] = va;
                Bs[kk][mm] = vb;
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < 16; ++kk) {
                T a[4], b[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
                for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int m = t.m0 + ty + 16 * i;
        if (m >= p.M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int n = t.n0 + tx + 16 * j;
            if (n >= p.N) continue;
            long long idx = p.c_off + (long long)m * p.scm + (long long)n * p.scn;
            T v = (T)p.alpha * acc[i][j];
            if (p.accumulate) v += C[idx];
            C[idx] = v;
        }
    }
}

// ------------------------------------------------------------------------------------------
// Block copies, MPO channel mixing, diagonal
// ------------------------------------------------------------------------------------------
// Arithmetic of an element-wise kernel: FP64 when it writes FP64, else FP32 (an FP32 or bf16 output
// cannot hold more; the FP64 pipe of this part is 1/64 of the FP32 one and would otherwise bound
// these memory-bound kernels).
template <class Tin, class Tout>
using ew_t = typename std::conditional<std::is_same<Tout, double>::value, double, float>::type;
template <class A, class T>
__device__ __forceinline__ A to_a(T x) { return (A)x; }
template <>
__device__ __forceinline__ float to_a<float, __nv_bfloat16>(__nv_bfloat16 x) { return __bfloat162float(x); }
template <>
__device__ __forceinline__ double to_a<double, __nv_bfloat16>(__nv_bfloat16 x) { return (double)__bfloat162float(x); }
template <class T, class A>
__device__ __forceinline__ T from_a(A v) { return (T)v; }
template <>
__device__ __forceinline__ __nv_bfloat16 from_a<__nv_bfloat16, float>(float v) { return __float2bfloat16_rn(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 from_a<__nv_bfloat16, double>(double v) { return __float2bfloat16_rn((float)v); }

// Element indices stay below 2^31 within a job (chunk starts are 32-bit), so the row/column split
// uses 32-bit division.
template <class Tin, class Tout>
__global__ void k_copy(const CopyJob* __restrict__ jobs, const int2* __restrict__ chunks, const Tin* __restrict__ src,
                       Tout* __restrict__ dst) {
    using A = ew_t<Tin, Tout>;
    const int2 ch = chunks[blockIdx.x];
    const CopyJob j = jobs[ch.x];
    const int w = j.cols > j.zero_to ? j.cols : j.zero_to;
    const long long total = (long long)j.rows * w;
    const int end = (int)min(total, (long long)ch.y + CHUNK);
    const A scale = (A)j.scale;
    for (int e = ch.y + (int)threadIdx.x; e < end; e += blockDim.x) {
        const int r = e / w, c = e - r * w;
        A v = A(0);
        if (c < j.cols) v = scale * to_a<A>(src[j.src + (long long)r * j.srs + (long long)c * j.scs]);
        dst[j.dst + (long long)r * j.drs + (long long)c * j.dcs] = from_a<Tout>(v);
    }
}

template <class Tin, class Tout>
__global__ void k_mix(const MixJob* __restrict__ jobs, const int2* __restrict__ chunks, const MixTerm* __restrict__ terms,
                      const Tin* __restrict__ in, Tout* __restrict__ out) {
    using A = ew_t<Tin, Tout>;
    const int2 ch = chunks[blockIdx.x];
    const MixJob j = jobs[ch.x];
    const int w = j.cols > j.zero_to ? j.cols : j.zero_to;
    const long long total = (long long)j.rows * w;
    const int end = (int)min(total, (long long)ch.y + CHUNK);
    for (int e = ch.y + (int)threadIdx.x; e < end; e += blockDim.x) {
        const int r = e / w, c = e - r * w;
        A v = A(0);
        if (c < j.cols) {
            for (int t = 0; t < j.nt; ++t) {
                const MixTerm tm = terms[j.t0 + t];
                v += (A)tm.coef * to_a<A>(in[tm.src + (long long)r * tm.ld + c]);
            }
        }
        out[j.dst + (long long)r * j.ldo + c] = from_a<Tout>(v);
    }
}

template <class T>
__global__ void k_diag(const DiagJob* __restrict__ jobs, const int2* __restrict__ chunks, const DiagTerm* __restrict__ terms,
                       const T* __restrict__ Ls, int ldl, const T* __restrict__ Rs, int ldr,
                       double* __restrict__ out) {
    const int2 ch = chunks[blockIdx.x];
    const DiagJob j = jobs[ch.x];
    const long long total = (long long)j.rows * j.cols;
    const long long end = min(total, (long long)ch.y + CHUNK);
    for (long long e = (long long)ch.y + threadIdx.x; e < end; e += blockDim.x) {
        int a = (int)(e / j.cols), c = (int)(e % j.cols);
        double v = 0.0;
        for (int t = 0; t < j.nt; ++t) {
            const DiagTerm tm = terms[j.t0 + t];
            v += tm.coef * to_d(Ls[tm.l + (long long)a * (ldl + 1)]) * to_d(Rs[tm.r + (long long)c * (ldr + 1)]);
        }
        out[j.off + e] = v;
    }
}

// ------------------------------------------------------------------------------------------
// Davidson vector kernels (FP64, deterministic two-pass reductions)
// ------------------------------------------------------------------------------------------
__global__ void k_dots_partial(const double* __restrict__ V, long long ldv, const double* __restrict__ y,
                               long long n, double* __restrict__ partial) {
    const int i = blockIdx.y, chunk = blockIdx.x, nchunks = gridDim.x;
    const long long per = (n + nchunks - 1) / nchunks;
    const long long b = chunk * per, e = min(n, b + per);
    double s = 0.0;
    for (long long x = b + threadIdx.x; x < e; x += blockDim.x) s = fma(V[i * ldv + x], y[x], s);
    s = block_sum(s);
    if (threadIdx.x == 0) partial[(long long)i * nchunks + chunk] = s;
}

__global__ void k_reduce_rows(const double* __restrict__ partial, int nchunks, double* __restrict__ out) {
    const int i = blockIdx.x;
    double s = 0.0;
    for (int c = threadIdx.x; c < nchunks; c += blockDim.x) s += partial[(long long)i * nchunks + c];
    s = block_sum(s);
    if (threadIdx.x == 0) out[i] = s;
}

// yth[0] = theta, yth[1..k] = Ritz coefficients.  norms[0] = |r|^2, norms[1] = |u|^2.
__global__ void k_ritz(const double* __restrict__ V, const double* __restrict__ AV, long long ldv,
                       int k, const double* __restrict__ yth, long long n, double* __restrict__ u,
                       double* __restrict__ Au, double* __restrict__ r, double* __restrict__ partial) {
    const int chunk = blockIdx.x, nchunks = gridDim.x;
    const long long per = (n + nchunks - 1) / nchunks;
    const long long b = chunk * per, e = min(n, b + per);
    const double th = yth[0];
    double sr = 0.0, su = 0.0;
    for (long long x = b + threadIdx.x; x < e; x += blockDim.x) {
        double uu = 0.0, aa = 0.0;
        for (int i = 0; i < k; ++i) {
            double yi = yth[1 + i];
            uu = fma(yi, V[i * ldv + x], uu);
            aa = fma(yi, AV[i * ldv + x], aa);
        }
        double rr = aa - th * uu;
        u[x] = uu;
        Au[x] = aa;
        r[x] = rr;
        sr = fma(rr, rr, sr);
        su = fma(uu, uu, su);
    }
    sr = block_sum(sr);
    su = block_sum(su);
    if (threadIdx.x == 0) {
        partial[chunk] = sr;
        partial[nchunks + chunk] = su;
    }
}

__global__ void k_precond(const double* __restrict__ r, const double* __restrict__ diag,
                          const double* __restrict__ theta, double fl, long long n, double* __restrict__ t) {
    const double th = theta[0];
    for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (long long)gridDim.x * blockDim.x) {
        double den = th - diag[x];
        if (fabs(den) < fl) den = den >= 0.0 ? fl : -fl;
        t[x] = r[x] / den;
    }
}

__global__ void k_subtract(const double* __restrict__ V, long long ldv, int k, const double* __restrict__ c,
                           long long n, double* __restrict__ t) {
    for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (long long)gridDim.x * blockDim.x) {
        double v = t[x];
        for (int i = 0; i < k; ++i) v = fma(-c[i], V[i * ldv + x], v);
        t[x] = v;
    }
}

__global__ void k_scale(const double* __restrict__ x, const double* __restrict__ nrm2, long long n,
                        double* __restrict__ y, int invert_sqrt) {
    const double s = invert_sqrt ? 1.0 / sqrt(nrm2[0]) : nrm2[0];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = x[i] * s;
}

__global__ void k_finite(const double* __restrict__ x, long long n, unsigned* err) {
    bool bad = false;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        if (!isfinite(x[i])) bad = true;
    if (bad) atomicOr(err, ERRBIT_NONFINITE);
}

// Lowest eigenpair of a small symmetric matrix (k <= 32) by cyclic Jacobi, one thread.
__global__ void k_small_eig(const double* __restrict__ G, int k, int ldg, double* __restrict__ yth) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double a[32][32], v[32][32];
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) {
            a[i][j] = 0.5 * (G[i * ldg + j] + G[j * ldg + i]);
            v[i][j] = (i == j) ? 1.0 : 0.0;
        }
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0, dia = 0.0;
        for (int i = 0; i < k; ++i) {
            dia += a[i][i] * a[i][i];
            for (int j = i + 1; j < k; ++j) off += a[i][j] * a[i][j];
        }
        if (off <= 1e-34 * dia || off == 0.0) break;
        for (int p = 0; p < k; ++p)
            for (int q = p + 1; q < k; ++q) {
                double apq = a[p][q];
                if (apq == 0.0) continue;
                double zeta = (a[q][q] - a[p][p]) / (2.0 * apq);
                double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
                for (int r = 0; r < k; ++r) {
                    double arp = a[r][p], arq = a[r][q];
                    a[r][p] = c * arp - s * arq;
                    a[r][q] = s * arp + c * arq;
                }
                for (int r = 0; r < k; ++r) {
                    double apr = a[p][r], aqr = a[q][r];
                    a[p][r] = c * apr - s * aqr;
                    a[q][r] = s * apr + c * aqr;
                }
                for (int r = 0; r < k; ++r) {
                    double vrp = v[r][p], vrq = v[r][q];
                    v[r][p] = c * vrp - s * vrq;
                    v[r][q] = s * vrp + c * vrq;
                }
            }
    }
    int best = 0;
    for (int i = 1; i < k; ++i)
        if (a[i][i] < a[best][best]) best = i;
    yth[0] = a[best][best];
    for (int i = 0; i < k; ++i) yth[1 + i] = v[i][best];
}

// ------------------------------------------------------------------------------------------
// One-sided Jacobi SVD (Hestenes).  W holds the sector matrix column-major (p x n, n <= p); pairs
// of columns are rotated until mutually orthogonal; V accumulates the rotations.  The rounds of
// a sweep follow the round-robin tournament (n/2 disjoint pairs per round, n-1 rounds).
// ------------------------------------------------------------------------------------------
template <class T>
__global__ void k_svd_init_v(const SvdSec* __restrict__ secs, T* __restrict__ V) {
    const SvdSec s = secs[blockIdx.y];
    const long long total = (long long)s.n * s.n;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        int c = (int)(e / s.n), r = (int)(e % s.n);
        V[s.v_off + e] = (r == c) ? T(1) : T(0);
    }
}

// Round-robin pairing: position 0 fixed, positions 1..npad-1 rotate by `round`.
__device__ __forceinline__ int rr_player(int pos, int round, int npad) {
    return pos == 0 ? 0 : ((pos - 1 + round) % (npad - 1)) + 1;
}

template <class T>
__device__ __forceinline__ T wsum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// One warp rotates one column pair; returns true if it rotated.  Each lane keeps its share of
// both columns (rows lane, lane+32, ...) in registers, so every phase costs one memory latency.
constexpr int JREG = 32;   // register-resident rows per lane: p and n up to 32*32 = 1024
template <class T>
__device__ __forceinline__ bool jacobi_pair(const SvdSec& s, int pi, int round, T* __restrict__ W,
                                            T* __restrict__ V, T tol, T floor_, int lane) {
    if (round >= s.npad - 1) return false;
    int i = rr_player(pi, round, s.npad);
    int j = rr_player(s.npad - 1 - pi, round, s.npad);
    if (i > j) { int t = i; i = j; j = t; }
    if (j >= s.n) return false;                      // bye against the padding column
    T* ci = W + s.w_off + (long long)i * s.p;
    T* cj = W + s.w_off + (long long)j * s.p;
    T* vi = V + s.v_off + (long long)i * s.n;
    T* vj = V + s.v_off + (long long)j * s.n;
    T al = 0, be = 0, ga = 0;
    if (s.p <= 32 * JREG && s.n <= 32 * JREG) {
        T x[JREG], y[JREG];
#pragma unroll
        for (int k = 0; k < JREG; ++k) {
            const int r = lane + 32 * k;
            x[k] = r < s.p ? ci[r] : T(0);
            y[k] = r < s.p ? cj[r] : T(0);
        }
#pragma unroll
        for (int k = 0; k < JREG; ++k) {
            al = fma(x[k], x[k], al);
            be = fma(y[k], y[k], be);
            ga = fma(x[k], y[k], ga);
        }
        al = wsum(al);
        be = wsum(be);
        ga = wsum(ga);
        if (ga == T(0) || !(fabs(ga) > tol * sqrt(al * be)) || fmin(al, be) <= floor_) return false;
        T zeta = (be - al) / (T(2) * ga);
        T t = (zeta >= T(0) ? T(1) : T(-1)) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
        T c = T(1) / sqrt(T(1) + t * t), sn = c * t;
        T u[JREG], w[JREG];
#pragma unroll
        for (int k = 0; k < JREG; ++k) {
            const int r = lane + 32 * k;
            u[k] = r < s.n ? vi[r] : T(0);
            w[k] = r < s.n ? vj[r] : T(0);
        }
#pragma unroll
        for (int k = 0; k < JREG; ++k) {
            const int r = lane + 32 * k;
            if (r < s.p) {
                ci[r] = c * x[k] - sn * y[k];
                cj[r] = sn * x[k] + c * y[k];
            }
            if (r < s.n) {
                vi[r] = c * u[k] - sn * w[k];
                vj[r] = sn * u[k] + c * w[k];
            }
        }
        return true;
    }
    for (int r = lane; r < s.p; r += 32) {
        T x = ci[r], y = cj[r];
        al = fma(x, x, al);
        be = fma(y, y, be);
        ga = fma(x, y, ga);
    }
    al = wsum(al);
    be = wsum(be);
    ga = wsum(ga);
    if (ga == T(0) || !(fabs(ga) > tol * sqrt(al * be)) || fmin(al, be) <= floor_) return false;
    T zeta = (be - al) / (T(2) * ga);
    T t = (zeta >= T(0) ? T(1) : T(-1)) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
    T c = T(1) / sqrt(T(1) + t * t), sn = c * t;
    for (int r = lane; r < s.p; r += 32) {
        T x = ci[r], y = cj[r];
        ci[r] = c * x - sn * y;
        cj[r] = sn * x + c * y;
    }
    for (int r = lane; r < s.n; r += 32) {
        T x = vi[r], y = vj[r];
        vi[r] = c * x - sn * y;
        vj[r] = sn * x + c * y;
    }
    return true;
}

// All sweeps of all sectors in one cooperative launch; bounded grid barrier between rounds.
// rot[sweep] counts the warps that rotated in that sweep (zeroed by the host); *sweeps = sweeps
// run; bar: 3 zeroed words for the barrier.
template <class T>
__global__ void k_jacobi_coop(const SvdSec* __restrict__ secs, const int* __restrict__ pair_sec, int npairs,
                              int maxnpad, int max_sweeps, T* __restrict__ W, T* __restrict__ V, T tol,
                              const double* __restrict__ floor2, int* __restrict__ rot, int* __restrict__ sweeps,
                              unsigned* __restrict__ bar, unsigned* __restrict__ err) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    int sweep = 0;
    bool alive = true;
    for (; sweep < max_sweeps && alive; ++sweep) {
        int mine = 0;
        for (int round = 0; round < maxnpad - 1 && alive; ++round) {
            for (int w = gw; w < npairs; w += nw) {
                const int si = pair_sec[w];
                const SvdSec s = secs[si];
                if (jacobi_pair<T>(s, w - s.pair0, round, W, V, tol * sqrt((T)s.p), floor2 ? (T)floor2[si] : T(0), lane)) mine = 1;
            }
            alive = grid_barrier(bar, gridDim.x, err);
        }
        if (!alive) break;
        if (lane == 0 && mine) atomicAdd(&rot[sweep], 1);
        alive = grid_barrier(bar, gridDim.x, err);
        if (!alive) break;
        if (*((volatile int*)&rot[sweep]) == 0) break;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *sweeps = sweep + 1;
}

// One round of one sweep of the scalar Jacobi (one warp per pair); rot[sweep] set when a pair
// rotated.  A launch whose previous sweep rotated nothing returns at once.
template <class T>
__global__ void k_jacobi_round(const SvdSec* __restrict__ secs, const int* __restrict__ pair_sec, int npairs,
                               int round, int sweep, T* __restrict__ W, T* __restrict__ V, T tol,
                               const double* __restrict__ floor2, int* __restrict__ rot) {
    if (sweep > 0 && *((volatile int*)&rot[sweep - 1]) == 0) return;
    const int lane = threadIdx.x & 31;
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= npairs) return;
    const int si = pair_sec[w];
    const SvdSec s = secs[si];
    if (jacobi_pair<T>(s, w - s.pair0, round, W, V, tol * sqrt((T)s.p), floor2 ? (T)floor2[si] : T(0), lane) && lane == 0)
        rot[sweep] = 1;
}

// floor2[s] = (eta * |W_s|_F)^2: columns below it are left unrotated (below working precision).
template <class T>
__global__ void k_svd_floor(const SvdSec* __restrict__ secs, const T* __restrict__ W, double eta,
                            double* __restrict__ floor2) {
    const SvdSec s = secs[blockIdx.x];
    double a = 0.0;
    const long long total = (long long)s.p * s.n;
    for (long long e = threadIdx.x; e < total; e += blockDim.x) {
        double x = (double)W[s.w_off + e];
        a = fma(x, x, a);
    }
    a = block_sum(a);
    if (threadIdx.x == 0) floor2[blockIdx.x] = eta * eta * a;
}

// sig[s_off + i] = |W_i| (FP64), order[s_off + r] = column with the r-th largest norm (ties: lower index).
template <class T>
__global__ void k_svd_finish(const SvdSec* __restrict__ secs, const T* __restrict__ W, double* __restrict__ sig,
                             int* __restrict__ order) {
    const SvdSec s = secs[blockIdx.x];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int c = wid; c < s.n; c += nw) {
        const T* col = W + s.w_off + (long long)c * s.p;
        double a = 0.0;
        for (int r = lane; r < s.p; r += 32) a = fma((double)col[r], (double)col[r], a);
        a = warp_sum(a);
        if (lane == 0) sig[s.s_off + c] = sqrt(a);
    }
    __syncthreads();
    for (int c = threadIdx.x; c < s.n; c += blockDim.x) {
        double v = sig[s.s_off + c];
        int rank = 0;
        for (int o = 0; o < s.n; ++o) {
            double w = sig[s.s_off + o];
            rank += (w > v) || (w == v && o < c);
        }
        order[s.s_off + rank] = c;
    }
}

// ------------------------------------------------------------------------------------------
// Truncation selection.  Keys (lambda desc, sector asc, position asc) over all sectors' values.
//   k_trunc_flat   flat arrays lam[g], sec[g], pos[g] (sector order, descending inside)
//   k_trunc_rank   rank of every candidate (lambda > rel_cutoff * lambda_max) among candidates
//   k_trunc_count  kept[s] and weights: total sum lambda^2, kept sum lambda^2
// ------------------------------------------------------------------------------------------
__global__ void k_trunc_flat(const SvdSec* __restrict__ secs, int nsec, const double* __restrict__ sig,
                             const int* __restrict__ order, double* __restrict__ lam, int* __restrict__ sec,
                             int* __restrict__ pos, double* __restrict__ lmax) {
    const int s = blockIdx.x;
    const SvdSec S = secs[s];
    double mx = 0.0;
    for (int i = threadIdx.x; i < S.n; i += blockDim.x) {
        double v = sig[S.s_off + order[S.s_off + i]];
        lam[S.s_off + i] = v;
        sec[S.s_off + i] = s;
        pos[S.s_off + i] = i;
        mx = fmax(mx, v);
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    __shared__ double red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
        lmax[s] = m;
    }
}

__global__ void k_trunc_rank(const double* __restrict__ lam, const int* __restrict__ sec, const int* __restrict__ pos,
                             int total, const double* __restrict__ lmax_sec, int nsec, double rel_cutoff,
                             int* __restrict__ rank) {
    __shared__ double thr_s;
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int s = 0; s < nsec; ++s) m = fmax(m, lmax_sec[s]);
        thr_s = rel_cutoff * m;
    }
    __syncthreads();
    const double thr = thr_s;
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= total) return;
    const double v = lam[g];
    const int sg = sec[g], pg = pos[g];
    int r = -1;
    if (v > thr) {
        r = 0;
        for (int o = 0; o < total; ++o) {
            const double w = lam[o];
            r += (w > thr) && ((w > v) || (w == v && (sec[o] < sg || (sec[o] == sg && pos[o] < pg))));
        }
    }
    rank[g] = r;
}

__global__ void __launch_bounds__(1024) k_trunc_count(const double* __restrict__ lam, const int* __restrict__ sec,
                                                      const int* __restrict__ rank, int total, int nsec, int m_max,
                                                      double degen_tol, int* __restrict__ kept,
                                                      double* __restrict__ weights) {
    __shared__ double s_next;
    __shared__ int s_cnt[256];
    if (threadIdx.x == 0) s_next = -1.0;
    for (int s = threadIdx.x; s < 256; s += blockDim.x) s_cnt[s] = 0;
    __syncthreads();
    double tot = 0.0;
    for (int g = threadIdx.x; g < total; g += blockDim.x) {
        tot += lam[g] * lam[g];
        if (rank[g] == m_max) s_next = lam[g];
    }
    tot = block_sum(tot);
    const double nxt = s_next;
    double kw = 0.0;
    for (int g = threadIdx.x; g < total; g += blockDim.x) {
        const int r = rank[g];
        const double a = lam[g];
        if (r >= 0 && r < m_max && (nxt < 0.0 || a > nxt * (1.0 + degen_tol))) {
            kw += a * a;
            atomicAdd(&s_cnt[sec[g]], 1);
        }
    }
    kw = block_sum(kw);
    for (int s = threadIdx.x; s < nsec; s += blockDim.x) kept[s] = s_cnt[s];
    if (threadIdx.x == 0) {
        weights[0] = tot;
        weights[1] = kw;
    }
}

inline int grid_for(long long elems, int cap = 4096) {
    long long g = (elems + 255) / 256;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

}  // namespace

// ------------------------------------------------------------------------------------------
// Launch wrappers
// ------------------------------------------------------------------------------------------
template <class T>
void launch_gemm_simt(const GProb* probs, const GSeg* segs, const GTile* tiles, int ntiles, const T* A, const T* B,
                      T* C, cudaStream_t st) {
    if (ntiles <= 0) return;
    k_gemm_simt<T><<<ntiles, 256, 0, st>>>(probs, segs, tiles, A, B, C);
    PD_LAUNCHED();
}
template void launch_gemm_simt<double>(const GProb*, const GSeg*, const GTile*, int, const double*, const double*,
                                       double*, cudaStream_t);
template void launch_gemm_simt<float>(const GProb*, const GSeg*, const GTile*, int, const float*, const float*,
                                      float*, cudaStream_t);

template <class Tin, class Tout>
void launch_copy(const CopyJob* jobs, const int2* chunks, int nchunks, const Tin* src, Tout* dst, cudaStream_t st) {
    if (nchunks <= 0) return;
    k_copy<Tin, Tout><<<nchunks, 256, 0, st>>>(jobs, chunks, src, dst);
    PD_LAUNCHED();
}

template <class Tin, class Tout>
void launch_mix(const MixJob* jobs, const int2* chunks, int nchunks, const MixTerm* terms, const Tin* in,
                Tout* out, cudaStream_t st) {
    if (nchunks <= 0) return;
    k_mix<Tin, Tout><<<nchunks, 256, 0, st>>>(jobs, chunks, terms, in, out);
    PD_LAUNCHED();
}

template <class T>
void launch_diag(const DiagJob* jobs, const int2* chunks, int nchunks, const DiagTerm* terms, const T* Ls, int ldl,
                 const T* Rs, int ldr, double* out, cudaStream_t st) {
    if (nchunks <= 0) return;
    k_diag<T><<<nchunks, 256, 0, st>>>(jobs, chunks, terms, Ls, ldl, Rs, ldr, out);
    PD_LAUNCHED();
}

template void launch_copy<double, double>(const CopyJob*, const int2*, int, const double*, double*, cudaStream_t);
template void launch_copy<double, float>(const CopyJob*, const int2*, int, const double*, float*, cudaStream_t);
template void launch_copy<double, __nv_bfloat16>(const CopyJob*, const int2*, int, const double*, __nv_bfloat16*, cudaStream_t);
template void launch_copy<float, double>(const CopyJob*, const int2*, int, const float*, double*, cudaStream_t);
template void launch_copy<float, float>(const CopyJob*, const int2*, int, const float*, float*, cudaStream_t);
template void launch_copy<float, __nv_bfloat16>(const CopyJob*, const int2*, int, const float*, __nv_bfloat16*, cudaStream_t);
template void launch_mix<double, double>(const MixJob*, const int2*, int, const MixTerm*, const double*, double*, cudaStream_t);
template void launch_mix<float, float>(const MixJob*, const int2*, int, const MixTerm*, const float*, float*, cudaStream_t);
template void launch_mix<float, __nv_bfloat16>(const MixJob*, const int2*, int, const MixTerm*, const float*, __nv_bfloat16*, cudaStream_t);
template void launch_diag<double>(const DiagJob*, const int2*, int, const DiagTerm*, const double*, int, const double*, int, double*, cudaStream_t);
template void launch_diag<float>(const DiagJob*, const int2*, int, const DiagTerm*, const float*, int, const float*, int, double*, cudaStream_t);

void launch_dots(const double* V, long long ldv, int k, const double* y, long long n, double* partial,
                 int nchunks, double* out, cudaStream_t st) {
    if (k <= 0) return;
    k_dots_partial<<<dim3(nchunks, k), 256, 0, st>>>(V, ldv, y, n, partial);
    PD_LAUNCHED();
    k_reduce_rows<<<k, 256, 0, st>>>(partial, nchunks, out);
    PD_LAUNCHED();
}

void launch_ritz(const double* V, const double* AV, long long ldv, int k, const double* yth, long long n,
                 double* u, double* Au, double* r, double* partial, int nchunks, double* norms, cudaStream_t st) {
    k_ritz<<<nchunks, 256, 0, st>>>(V, AV, ldv, k, yth, n, u, Au, r, partial);
    PD_LAUNCHED();
    k_reduce_rows<<<2, 256, 0, st>>>(partial, nchunks, norms);
    PD_LAUNCHED();
}

void launch_precond(const double* r, const double* diag, const double* theta, double fl, long long n,
                    double* t, cudaStream_t st) {
    k_precond<<<grid_for(n), 256, 0, st>>>(r, diag, theta, fl, n, t);
    PD_LAUNCHED();
}

void launch_subtract(const double* V, long long ldv, int k, const double* c, long long n, double* t,
                     cudaStream_t st) {
    k_subtract<<<grid_for(n), 256, 0, st>>>(V, ldv, k, c, n, t);
    PD_LAUNCHED();
}

void launch_scale(const double* x, const double* nrm2, long long n, double* y, int invert_sqrt, cudaStream_t st) {
    k_scale<<<grid_for(n), 256, 0, st>>>(x, nrm2, n, y, invert_sqrt);
    PD_LAUNCHED();
}

void launch_small_eig(const double* G, int k, int ldg, double* yth, cudaStream_t st) {
    PD_REQUIRE(k >= 1 && k <= 32, DMRG_ERR_CAPACITY, "Davidson subspace larger than 32");
    k_small_eig<<<1, 32, 0, st>>>(G, k, ldg, yth);
    PD_LAUNCHED();
}

void launch_nrm2(const double* x, long long n, double* partial, int nchunks, double* out, cudaStream_t st) {
    launch_dots(x, 0, 1, x, n, partial, nchunks, out, st);
}

void launch_finite_check(const double* x, long long n, unsigned* err, cudaStream_t st) {
    k_finite<<<grid_for(n, 1024), 256, 0, st>>>(x, n, err);
    PD_LAUNCHED();
}

template <class T>
void launch_svd_init_v(const SvdSec* secs, int nsec, int max_n, T* V, cudaStream_t st) {
    if (nsec <= 0) return;
    k_svd_init_v<T><<<dim3(grid_for((long long)max_n * max_n, 256), nsec), 256, 0, st>>>(secs, V);
    PD_LAUNCHED();
}
template void launch_svd_init_v<double>(const SvdSec*, int, int, double*, cudaStream_t);
template void launch_svd_init_v<float>(const SvdSec*, int, int, float*, cudaStream_t);

template <class T>
void launch_jacobi(const SvdSec* secs, int nsec, const int* pair_sec, int npairs, int maxnpad, int max_sweeps, T* W,
                   T* V, T tol, double eta, double* floor2, int* rot, int* sweeps, unsigned* bar, unsigned* err,
                   cudaStream_t st) {
    if (npairs <= 0 || maxnpad < 2) return;
    const double* fl = nullptr;
    if (eta > 0.0) {
        k_svd_floor<T><<<nsec, 256, 0, st>>>(secs, W, eta, floor2);
        PD_LAUNCHED();
        fl = floor2;
    }
    const int threads = 128;   // register-heavy pair updates: small blocks keep several per SM
    if (g_sm_cap > 0) {
        // regions run concurrently: one launch per round (no grid barrier spinning on SMs that
        // other regions' kernels need), convergence read one sweep behind
        const int grid = (npairs * 32 + threads - 1) / threads;
        int* hrot = sweep_flags_host(max_sweeps);
        std::vector<cudaEvent_t> evs(max_sweeps, nullptr);
        int done = max_sweeps;
        auto cleanup = [&]() {
            for (auto e : evs)
                if (e) cudaEventDestroy(e);
        };
        try {
            for (int sweep = 0; sweep < max_sweeps; ++sweep) {
                for (int round = 0; round < maxnpad - 1; ++round) {
                    k_jacobi_round<T><<<grid, threads, 0, st>>>(secs, pair_sec, npairs, round, sweep, W, V, tol, fl,
                                                                rot);
                    PD_LAUNCHED();
                }
                PD_CK(cudaMemcpyAsync(hrot + sweep, rot + sweep, sizeof(int), cudaMemcpyDeviceToHost, st));
                PD_CK(cudaEventCreateWithFlags(&evs[sweep], cudaEventDisableTiming));
                PD_CK(cudaEventRecord(evs[sweep], st));
                if (sweep > 0) {
                    PD_CK(cudaEventSynchronize(evs[sweep - 1]));
                    if (hrot[sweep - 1] == 0) {
                        done = sweep;
                        break;
                    }
                }
            }
        } catch (...) {
            cleanup();
            throw;
        }
        cleanup();
        PD_CK(cudaMemcpyAsync(sweeps, &done, sizeof(int), cudaMemcpyHostToDevice, st));
        return;
    }
    static int per_sm[2] = {0, 0};
    int& ps = per_sm[sizeof(T) == 8 ? 1 : 0];
    if (!ps) PD_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ps, k_jacobi_coop<T>, threads, 0));
    int dev = 0, sms = 0;
    PD_CK(cudaGetDevice(&dev));
    PD_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int need = (npairs * 32 + threads - 1) / threads;
    int blocks = std::max(1, std::min(need, ps * sm_share(sms)));
    PD_CK(cudaMemsetAsync(bar, 0, 3 * sizeof(unsigned), st));
    void* args[] = {(void*)&secs, (void*)&pair_sec, (void*)&npairs, (void*)&maxnpad, (void*)&max_sweeps,
                    (void*)&W, (void*)&V, (void*)&tol, (void*)&fl, (void*)&rot, (void*)&sweeps, (void*)&bar,
                    (void*)&err};
    PD_CK(cudaLaunchCooperativeKernel((void*)k_jacobi_coop<T>, blocks, threads, args, 0, st));
    PD_LAUNCHED();
}
template void launch_jacobi<double>(const SvdSec*, int, const int*, int, int, int, double*, double*, double, double,
                                    double*, int*, int*, unsigned*, unsigned*, cudaStream_t);
template void launch_jacobi<float>(const SvdSec*, int, const int*, int, int, int, float*, float*, float, double,
                                   double*, int*, int*, unsigned*, unsigned*, cudaStream_t);

template <class T>
void launch_svd_finish(const SvdSec* secs, int nsec, const T* W, double* sig, int* order, cudaStream_t st) {
    if (nsec <= 0) return;
    k_svd_finish<T><<<nsec, 256, 0, st>>>(secs, W, sig, order);
    PD_LAUNCHED();
}
template void launch_svd_finish<double>(const SvdSec*, int, const double*, double*, int*, cudaStream_t);
template void launch_svd_finish<float>(const SvdSec*, int, const float*, double*, int*, cudaStream_t);

void launch_truncate(const SvdSec* secs, int nsec, const double* sig, const int* order, int total, int m_max,
                     double rel_cutoff, double degen_tol, int* kept, double* weights, double* scratch_d, int* scratch_i,
                     cudaStream_t st) {
    PD_REQUIRE(nsec <= 256, DMRG_ERR_CAPACITY, "more than 256 charge sectors on one bond");
    if (total <= 0) return;
    double* lam = scratch_d;
    double* lmax = scratch_d + total;
    int* sec = scratch_i;
    int* pos = scratch_i + total;
    int* rank = scratch_i + 2 * total;
    k_trunc_flat<<<nsec, 256, 0, st>>>(secs, nsec, sig, order, lam, sec, pos, lmax);
    PD_LAUNCHED();
    k_trunc_rank<<<(total + 127) / 128, 128, 0, st>>>(lam, sec, pos, total, lmax, nsec, rel_cutoff, rank);
    PD_LAUNCHED();
    k_trunc_count<<<1, 1024, 0, st>>>(lam, sec, rank, total, nsec, m_max, degen_tol, kept, weights);
    PD_LAUNCHED();
}

}  // namespace pd
