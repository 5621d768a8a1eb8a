// FP64 / memory-bound kernels of the two-site DMRG step.
//
//  * k_gemm64       grouped, strided FP64 GEMM (the parity-mode contractions of the projected
//                   Hamiltonian and of the projected-operator updates, Sec. II)
//  * k_copy/k_mix   block gathers, transposes, MPO channel mixing (memory-bound)
//  * k_diag         diagonal of the projected Hamiltonian (Davidson preconditioner)
//  * Davidson       dot products, Ritz vectors, residuals, Gram-Schmidt, small Jacobi eigensolver
//  * SVD            batched one-sided (Hestenes) Jacobi SVD per charge sector, Eq. (svd)
//  * truncation     global keep-largest-m selection over all sectors (single CTA)
#include <cfloat>
#include <cmath>

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
// Grouped FP64 GEMM: 64x64 output tile per CTA, 256 threads, 4x4 per thread, K chunks of 16.
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_gemm64(const GProb* __restrict__ probs,
                                                const GSeg* __restrict__ segs,
                                                const GTile* __restrict__ tiles,
                                                const double* __restrict__ A,
                                                const double* __restrict__ B,
                                                double* __restrict__ C) {
    __shared__ double As[16][65];
    __shared__ double Bs[16][65];
    const GTile t = tiles[blockIdx.x];
    const GProb p = probs[t.prob];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    for (int sgi = 0; sgi < p.nseg; ++sgi) {
        const GSeg sg = segs[p.seg0 + sgi];
        for (int k0 = 0; k0 < sg.K; k0 += 16) {
            for (int e = tid; e < 1024; e += 256) {
                int kk = e & 15, mm = e >> 4;
                int m = t.m0 + mm, k = k0 + kk;
                double va = 0.0, vb = 0.0;
                if (m < p.M && k < sg.K) va = A[sg.a_off + (long long)m * p.sam + (long long)k * p.sak];
                int n = t.n0 + mm;
                if (n < p.N && k < sg.K) vb = B[sg.b_off + (long long)n * p.sbn + (long long)k * p.sbk];
                As[kk][mm] = va;
                Bs[kk][mm] = vb;
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < 16; ++kk) {
                double a[4], b[4];
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
            double v = p.alpha * acc[i][j];
            if (p.accumulate) v += C[idx];
            C[idx] = v;
        }
    }
}

// ------------------------------------------------------------------------------------------
// Block copies, MPO channel mixing, diagonal
// ------------------------------------------------------------------------------------------
template <class Tin, class Tout>
__global__ void k_copy(const CopyJob* __restrict__ jobs, const Tin* __restrict__ src,
                       Tout* __restrict__ dst) {
    const CopyJob j = jobs[blockIdx.y];
    const int w = j.cols > j.zero_to ? j.cols : j.zero_to;
    const long long total = (long long)j.rows * w;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        int r = (int)(e / w), c = (int)(e % w);
        double v = 0.0;
        if (c < j.cols) v = j.scale * to_d(src[j.src + (long long)r * j.srs + (long long)c * j.scs]);
        dst[j.dst + (long long)r * j.drs + (long long)c * j.dcs] = from_d<Tout>(v);
    }
}

template <class Tin, class Tout>
__global__ void k_mix(const MixJob* __restrict__ jobs, const MixTerm* __restrict__ terms,
                      const Tin* __restrict__ in, Tout* __restrict__ out) {
    const MixJob j = jobs[blockIdx.y];
    const int w = j.cols > j.zero_to ? j.cols : j.zero_to;
    const long long total = (long long)j.rows * w;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        int r = (int)(e / w), c = (int)(e % w);
        double v = 0.0;
        if (c < j.cols) {
            for (int t = 0; t < j.nt; ++t) {
                const MixTerm tm = terms[j.t0 + t];
                v += tm.coef * to_d(in[tm.src + (long long)r * tm.ld + c]);
            }
        }
        out[j.dst + (long long)r * j.ldo + c] = from_d<Tout>(v);
    }
}

template <class T>
__global__ void k_diag(const DiagJob* __restrict__ jobs, const DiagTerm* __restrict__ terms,
                       const T* __restrict__ Ls, int ldl, const T* __restrict__ Rs, int ldr,
                       double* __restrict__ out) {
    const DiagJob j = jobs[blockIdx.y];
    const long long total = (long long)j.rows * j.cols;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
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
// One-sided Jacobi SVD
// ------------------------------------------------------------------------------------------
__global__ void k_svd_init_v(const SvdSec* __restrict__ secs, double* __restrict__ V) {
    const SvdSec s = secs[blockIdx.y];
    const long long total = (long long)s.n * s.n;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        int c = (int)(e / s.n), r = (int)(e % s.n);
        V[s.v_off + e] = (r == c) ? 1.0 : 0.0;
    }
}

// Round-robin pairing: position 0 fixed, positions 1..npad-1 rotate by `round`.
__device__ __forceinline__ int rr_player(int pos, int round, int npad) {
    return pos == 0 ? 0 : ((pos - 1 + round) % (npad - 1)) + 1;
}

__global__ void k_jacobi_round(const SvdSec* __restrict__ secs, const int* __restrict__ pair_sec,
                               int npairs, int round, double* __restrict__ W, double* __restrict__ V,
                               double tol, int* __restrict__ rotated) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= npairs) return;
    const int si = pair_sec[warp];
    const SvdSec s = secs[si];
    const int pi = warp - s.pair0;
    if (round >= s.npad - 1) return;
    int i = rr_player(pi, round, s.npad);
    int j = rr_player(s.npad - 1 - pi, round, s.npad);
    if (i > j) { int t = i; i = j; j = t; }
    if (j >= s.n) return;                      // bye against the padding column
    double* ci = W + s.w_off + (long long)i * s.p;
    double* cj = W + s.w_off + (long long)j * s.p;
    double al = 0.0, be = 0.0, ga = 0.0;
    for (int r = lane; r < s.p; r += 32) {
        double x = ci[r], y = cj[r];
        al = fma(x, x, al);
        be = fma(y, y, be);
        ga = fma(x, y, ga);
    }
    al = warp_sum(al);
    be = warp_sum(be);
    ga = warp_sum(ga);
    if (ga == 0.0 || !(fabs(ga) > tol * sqrt(al * be))) return;
    double zeta = (be - al) / (2.0 * ga);
    double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
    double c = 1.0 / sqrt(1.0 + t * t), sn = c * t;
    for (int r = lane; r < s.p; r += 32) {
        double x = ci[r], y = cj[r];
        ci[r] = c * x - sn * y;
        cj[r] = sn * x + c * y;
    }
    double* vi = V + s.v_off + (long long)i * s.n;
    double* vj = V + s.v_off + (long long)j * s.n;
    for (int r = lane; r < s.n; r += 32) {
        double x = vi[r], y = vj[r];
        vi[r] = c * x - sn * y;
        vj[r] = sn * x + c * y;
    }
    if (lane == 0) atomicOr(rotated, 1);
}

// sig[s_off + i] = |W_i|, order[s_off + r] = column with the r-th largest norm (ties: lower index).
__global__ void k_svd_finish(const SvdSec* __restrict__ secs, const double* __restrict__ W,
                             double* __restrict__ sig, int* __restrict__ order) {
    const SvdSec s = secs[blockIdx.x];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int c = wid; c < s.n; c += nw) {
        const double* col = W + s.w_off + (long long)c * s.p;
        double a = 0.0;
        for (int r = lane; r < s.p; r += 32) a = fma(col[r], col[r], a);
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
// Truncation selection (one CTA).  Keys (lambda desc, sector asc, position asc).
// kept[s] = kept count of sector s; weights[0] = total sum lambda^2, weights[1] = kept sum.
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_truncate(const SvdSec* __restrict__ secs, int nsec,
                                                   const double* __restrict__ sig, const int* __restrict__ order,
                                                   int total, int m_max, double rel_cutoff, double degen_tol,
                                                   int* __restrict__ kept, double* __restrict__ weights) {
    extern __shared__ unsigned char smem[];
    double* lam = reinterpret_cast<double*>(smem);
    int* sec = reinterpret_cast<int*>(lam + total);
    int* pos = sec + total;
    int* rk = pos + total;
    __shared__ double s_lmax, s_next;
    __shared__ int s_kept_cnt[256];
    __shared__ double red[32];
    // flatten: sector s occupies [s_off, s_off + n) (sectors packed back to back)
    for (int s = 0; s < nsec; ++s) {
        const SvdSec S = secs[s];
        for (int i = threadIdx.x; i < S.n; i += blockDim.x) {
            lam[S.s_off + i] = sig[S.s_off + order[S.s_off + i]];
            sec[S.s_off + i] = s;
            pos[S.s_off + i] = i;
        }
    }
    for (int s = threadIdx.x; s < 256; s += blockDim.x) s_kept_cnt[s] = 0;
    __syncthreads();
    double mx = 0.0, tot = 0.0;
    for (int g = threadIdx.x; g < total; g += blockDim.x) {
        mx = fmax(mx, lam[g]);
        tot += lam[g] * lam[g];
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
        s_lmax = m;
        s_next = -1.0;
    }
    tot = block_sum(tot);          // contains __syncthreads, s_lmax visible afterwards
    const double thr = rel_cutoff * s_lmax;
    for (int g = threadIdx.x; g < total; g += blockDim.x) {
        const double v = lam[g];
        int rank = -1;
        if (v > thr) {
            rank = 0;
            for (int o = 0; o < total; ++o) {
                const double w = lam[o];
                if (!(w > thr)) continue;
                rank += (w > v) || (w == v && (sec[o] < sec[g] || (sec[o] == sec[g] && pos[o] < pos[g])));
            }
            if (rank == m_max) s_next = v;
        }
        rk[g] = rank;
    }
    __syncthreads();
    const double nxt = s_next;
    double kw = 0.0;
    for (int g = threadIdx.x; g < total; g += blockDim.x) {
        const int r = rk[g];
        const double a = lam[g];
        if (r >= 0 && r < m_max && (nxt < 0.0 || a > nxt * (1.0 + degen_tol))) {
            kw += a * a;
            atomicAdd(&s_kept_cnt[sec[g]], 1);
        }
    }
    kw = block_sum(kw);
    for (int s = threadIdx.x; s < nsec; s += blockDim.x) kept[s] = s_kept_cnt[s];
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
void launch_gemm64(const GProb* probs, const GSeg* segs, const GTile* tiles, int ntiles,
                   const double* A, const double* B, double* C, cudaStream_t st) {
    if (ntiles <= 0) return;
    k_gemm64<<<ntiles, 256, 0, st>>>(probs, segs, tiles, A, B, C);
    PD_LAUNCHED();
}

template <class Tin, class Tout>
void launch_copy(const CopyJob* jobs, int njobs, int max_elems, const Tin* src, Tout* dst, cudaStream_t st) {
    if (njobs <= 0) return;
    PD_REQUIRE(njobs <= 65535, DMRG_ERR_CAPACITY, "too many copy jobs in one launch");
    dim3 g(grid_for(max_elems, 512), njobs);
    k_copy<Tin, Tout><<<g, 256, 0, st>>>(jobs, src, dst);
    PD_LAUNCHED();
}

template <class Tin, class Tout>
void launch_mix(const MixJob* jobs, int njobs, int max_elems, const MixTerm* terms, const Tin* in,
                Tout* out, cudaStream_t st) {
    if (njobs <= 0) return;
    PD_REQUIRE(njobs <= 65535, DMRG_ERR_CAPACITY, "too many mix jobs in one launch");
    dim3 g(grid_for(max_elems, 512), njobs);
    k_mix<Tin, Tout><<<g, 256, 0, st>>>(jobs, terms, in, out);
    PD_LAUNCHED();
}

template <class T>
void launch_diag(const DiagJob* jobs, int njobs, int max_elems, const DiagTerm* terms, const T* Ls, int ldl,
                 const T* Rs, int ldr, double* out, cudaStream_t st) {
    if (njobs <= 0) return;
    PD_REQUIRE(njobs <= 65535, DMRG_ERR_CAPACITY, "too many diagonal jobs in one launch");
    dim3 g(grid_for(max_elems, 512), njobs);
    k_diag<T><<<g, 256, 0, st>>>(jobs, terms, Ls, ldl, Rs, ldr, out);
    PD_LAUNCHED();
}

template void launch_copy<double, double>(const CopyJob*, int, int, const double*, double*, cudaStream_t);
template void launch_copy<double, float>(const CopyJob*, int, int, const double*, float*, cudaStream_t);
template void launch_copy<double, __nv_bfloat16>(const CopyJob*, int, int, const double*, __nv_bfloat16*, cudaStream_t);
template void launch_copy<float, double>(const CopyJob*, int, int, const float*, double*, cudaStream_t);
template void launch_copy<float, float>(const CopyJob*, int, int, const float*, float*, cudaStream_t);
template void launch_copy<float, __nv_bfloat16>(const CopyJob*, int, int, const float*, __nv_bfloat16*, cudaStream_t);
template void launch_mix<double, double>(const MixJob*, int, int, const MixTerm*, const double*, double*, cudaStream_t);
template void launch_mix<float, float>(const MixJob*, int, int, const MixTerm*, const float*, float*, cudaStream_t);
template void launch_mix<float, __nv_bfloat16>(const MixJob*, int, int, const MixTerm*, const float*, __nv_bfloat16*, cudaStream_t);
template void launch_diag<double>(const DiagJob*, int, int, const DiagTerm*, const double*, int, const double*, int, double*, cudaStream_t);
template void launch_diag<float>(const DiagJob*, int, int, const DiagTerm*, const float*, int, const float*, int, double*, cudaStream_t);

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

void launch_svd_init_v(const SvdSec* secs, int nsec, int max_n, double* V, cudaStream_t st) {
    if (nsec <= 0) return;
    k_svd_init_v<<<dim3(grid_for((long long)max_n * max_n, 256), nsec), 256, 0, st>>>(secs, V);
    PD_LAUNCHED();
}

void launch_jacobi_round(const SvdSec* secs, const int* pair_sec, int npairs, int round, double* W, double* V,
                         double tol, int* rotated, cudaStream_t st) {
    if (npairs <= 0) return;
    int warps_per_block = 8;
    int blocks = (npairs + warps_per_block - 1) / warps_per_block;
    k_jacobi_round<<<blocks, 32 * warps_per_block, 0, st>>>(secs, pair_sec, npairs, round, W, V, tol, rotated);
    PD_LAUNCHED();
}

void launch_svd_finish(const SvdSec* secs, int nsec, int max_n, const double* W, double* sig, int* order,
                       cudaStream_t st) {
    if (nsec <= 0) return;
    (void)max_n;
    k_svd_finish<<<nsec, 256, 0, st>>>(secs, W, sig, order);
    PD_LAUNCHED();
}

void launch_truncate(const SvdSec* secs, int nsec, const double* sig, const int* order, int total, int m_max,
                     double rel_cutoff, double degen_tol, int* kept, double* weights, cudaStream_t st) {
    PD_REQUIRE(nsec <= 256, DMRG_ERR_CAPACITY, "more than 256 charge sectors on one bond");
    PD_REQUIRE(total <= 10000, DMRG_ERR_CAPACITY, "more than 10000 singular values on one bond");
    size_t smem = (size_t)total * (sizeof(double) + 3 * sizeof(int)) + 16;
    if (smem > 48 * 1024)
        PD_CK(cudaFuncSetAttribute(k_truncate, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_truncate<<<1, 1024, smem, st>>>(secs, nsec, sig, order, total, m_max, rel_cutoff, degen_tol, kept, weights);
    PD_LAUNCHED();
}

}  // namespace pd
