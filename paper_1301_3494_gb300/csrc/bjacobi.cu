// Block one-sided Jacobi SVD in FP32 for the charge sectors of the two-site wavefunction
// (the decomposition of Eq. (svd), Sec. II).
//
// The columns of every sector matrix W (p x n, column-major, n <= p) are cut into blocks of 16.
// A sweep pairs every block with every other block once (round-robin ordering of the blocks);
// a round processes all pairs of all sectors at once, one pair per CTA.  With the GPU to itself
// the caller runs all sweeps in one cooperative launch (a bounded grid barrier ends each round);
// while regions run concurrently, each round is its own launch (kernel boundaries order the
// rounds and nothing spins, so the regions' kernels interleave freely).  For a pair (I, J), I < J, the CTA stages the p x 32 columns in shared memory,
// forms their 32 x 32 Gram matrix, diagonalises it with a few sweeps of two-sided cyclic
// Jacobi, orders the eigenvectors by decreasing eigenvalue (block I receives the larger ones),
// and rotates the staged columns and the matching columns of V by that orthogonal matrix.  The
// sector has converged when a sweep finds no pair to rotate; the test of a pair is computed from
// the current columns, so the inexact inner solve is corrected by the next visit.
//
// Compared with rotating single column pairs, the number of grid-wide synchronisations per
// sweep drops from n - 1 to n / 16 - 1, and the work of a round becomes dense (Gram matrix and
// a 32-column rotation per CTA).
//
// A pair of columns (u, v) is rotated when |g_uv| > tol * |w_u| |w_v| + noise * (|w_u| + |w_v|),
// with noise = c * eps_f32 * sigma_max: the second term is the absolute rounding level of FP32
// columns of a matrix whose largest singular value is sigma_max.  Pairs below it are left as
// they are; their effect on the kept weight is below eps_f32 * sigma_max^2.
//
// Unchanged pairs are skipped: every block records the time (sweep * rounds + round + 1) it was
// last rotated, every block pair the time it was last found converged; a pair found converged
// after both of its blocks' last rotations has the same Gram matrix as then (and the noise level
// only grows), so it is converged still and is not staged again.  In a round a block belongs to
// one pair only, so each stamp has one writer per round; they are read after the round's grid
// barrier (or kernel boundary), from L2.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <vector>

#include "grid_sync.cuh"
#include "internal.h"

namespace pd {

namespace {

constexpr int BJ_B = 16;                     // columns per block
constexpr int BJ_K = 2 * BJ_B;               // columns of a block pair (= warp width)
constexpr int BJ_NP = BJ_K / 2;              // column pairs per inner round
constexpr int BJ_LD = BJ_K + 1;              // row stride of staged rows (conflict-free)
constexpr int BJ_QLD = BJ_K + 4;             // row stride of rotations (16-byte aligned rows)
constexpr int BJ_THREADS = 256;
constexpr int BJ_WARPS = BJ_THREADS / 32;
constexpr int BJ_SMEM_MAX = 226 * 1024;        // dynamic shared memory ceiling (227 KB less static use)

struct alignas(16) BjShared {
    float G[BJ_K * BJ_LD];             // Gram matrix (rotated in place)
    float Q[2][BJ_K * BJ_QLD];         // accumulated rotation; its column-permuted copy
    float Gp[BJ_WARPS][BJ_K * BJ_K];   // per-warp partial Gram matrices
    float c[BJ_NP], s[BJ_NP];          // rotation of each pair of the current inner round
    float diag[BJ_K];
    int gcol[BJ_K];                    // sector column of staged column u (-1: padding)
    int perm[BJ_K];                    // perm[r] = eigenvector placed at position r
    unsigned char lo[BJ_K - 1][BJ_NP], hi[BJ_K - 1][BJ_NP];   // inner round-robin pairs
    float noise;
    int flag[2];                       // any rotation in the inner round (by round parity)
    int qitem, qok;                    // work queue: item taken by this CTA, its state
};
static_assert(sizeof(BjShared) % 16 == 0, "staging area must stay 16-byte aligned");

__device__ __forceinline__ int rr_pos(int pos, int round, int npad) {
    return pos == 0 ? 0 : ((pos - 1 + round) % (npad - 1)) + 1;
}

__device__ __forceinline__ bool bj_need(float guv, float guu, float gvv, float tol, float noise) {
    if (!(guu > 0.f) || !(gvv > 0.f)) return false;
    const float su = guu * rsqrtf(guu), sv = gvv * rsqrtf(gvv);   // approximate roots: a threshold
    return fabsf(guv) > tol * su * sv + noise * (su + sv);
}

__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// X[r][u] = src[gcol[u] * ld + r0 + r] for r < rows (zero for padding columns), as asynchronous
// copies (the caller commits and waits).
__device__ __forceinline__ void bj_stage_async(float* __restrict__ X, const float* __restrict__ src, int ld, int r0,
                                               int rows, const int* __restrict__ gcol) {
    for (int u = 0; u < BJ_K; ++u) {
        const int c = gcol[u];
        if (c >= 0) {
            const float* col = src + (long long)c * ld + r0;
            for (int r = threadIdx.x; r < rows; r += BJ_THREADS) cp_async4(X + r * BJ_LD + u, col + r);
        } else {
            for (int r = threadIdx.x; r < rows; r += BJ_THREADS) X[r * BJ_LD + u] = 0.f;
        }
    }
}

// dst[gcol[u] * ld + r0 + r] = X[r][u] for u < k, r < rows: a thread reads a whole staged row,
// then stores it to the k columns (coalesced across the warp).
__device__ __forceinline__ void bj_unstage(const float* __restrict__ X, float* __restrict__ dst, int ld, int r0,
                                           int rows, const int* __restrict__ gcol, int k) {
    int cols[BJ_K];
#pragma unroll
    for (int u = 0; u < BJ_K; ++u) cols[u] = gcol[u];
    for (int r = threadIdx.x; r < rows; r += BJ_THREADS) {
        float v[BJ_K];
#pragma unroll
        for (int u = 0; u < BJ_K; ++u) v[u] = X[r * BJ_LD + u];
#pragma unroll
        for (int u = 0; u < BJ_K; ++u)
            if (u < k) dst[(long long)cols[u] * ld + r0 + r] = v[u];
    }
}

// Gram accumulation over `rows` staged rows into a lane's 8 x 8 tile (one of two interleaved row
// halves of the warp's rows); bj_gram_reduce then sums halves by shuffle and warps in warp order
// into S.G.
__device__ __forceinline__ void bj_gram_acc(float (&acc)[8][8], const float* __restrict__ X, int rows) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int u0 = 8 * (lane & 3), v0 = 8 * ((lane >> 2) & 3), half = lane >> 4;
    for (int r = 2 * w + half; r < rows; r += 2 * BJ_WARPS) {
        const float* xr = X + r * BJ_LD;
        float a[8], b[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) a[i] = xr[u0 + i];
#pragma unroll
        for (int j = 0; j < 8; ++j) b[j] = xr[v0 + j];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
}

__device__ __forceinline__ void bj_gram_reduce(BjShared& S, float (&acc)[8][8]) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int u0 = 8 * (lane & 3), v0 = 8 * ((lane >> 2) & 3), half = lane >> 4;
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] += __shfl_xor_sync(0xffffffffu, acc[i][j], 16);
    if (half == 0) {
        float* gp = S.Gp[w];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) gp[(u0 + i) * BJ_K + v0 + j] = acc[i][j];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < BJ_K * BJ_K; e += BJ_THREADS) {
        float g = 0.f;
#pragma unroll
        for (int ww = 0; ww < BJ_WARPS; ++ww) g += S.Gp[ww][e];
        S.G[(e >> 5) * BJ_LD + (e & 31)] = g;
    }
}

// X <- X Qp in place over `rows` staged rows.  Lane: 8 output columns of 4 rows; a warp owns
// 32 consecutive rows per pass.
__device__ __forceinline__ void bj_rotate(float* __restrict__ X, const float* __restrict__ Qp, int rows) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int c0 = 8 * (lane & 3), rg = lane >> 2;
    for (int rb = w * 32; rb < rows; rb += BJ_WARPS * 32) {
        int r[4];
        bool ok[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            r[i] = rb + rg + 8 * i;
            ok[i] = r[i] < rows;
        }
        float acc[4][8];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
#pragma unroll 4
        for (int u = 0; u < BJ_K; ++u) {
            float x[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) x[i] = ok[i] ? X[r[i] * BJ_LD + u] : 0.f;
            const float4 qa = *reinterpret_cast<const float4*>(Qp + u * BJ_QLD + c0);
            const float4 qb = *reinterpret_cast<const float4*>(Qp + u * BJ_QLD + c0 + 4);
            const float q[8] = {qa.x, qa.y, qa.z, qa.w, qb.x, qb.y, qb.z, qb.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(x[i], q[j], acc[i][j]);
        }
        __syncwarp();
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (ok[i])
#pragma unroll
                for (int j = 0; j < 8; ++j) X[r[i] * BJ_LD + c0 + j] = acc[i][j];
        __syncwarp();
    }
}

// Rotation (c, s) annihilating g_pq of the pair (p, q): new_p = c p - s q, new_q = s p + c q.
// The angle may be slightly inexact (fast reciprocals; the next visit corrects it), but c and s
// are normalised to c^2 + s^2 = 1 within an ulp (one Newton step on the reciprocal root), since
// the accumulated rotations must stay orthogonal.
__device__ __forceinline__ void bj_rot(float gpp, float gqq, float gpq, float& c, float& s) {
    const float zeta = __fdividef(gqq - gpp, 2.f * gpq);
    const float az = fabsf(zeta);
    // t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)); for huge |zeta|, t ~ 1 / (2 zeta)
    float t = az < 1e18f ? __fdividef(1.f, az + sqrtf(fmaf(az, az, 1.f))) : __fdividef(0.5f, az);
    t = zeta >= 0.f ? t : -t;
    const float x = fmaf(t, t, 1.f);
    float y = rsqrtf(x);
    y = y * fmaf(-0.5f * x * y, y, 1.5f);
    c = y;
    s = y * t;
}

// Two-sided cyclic Jacobi on the Gram matrix S.G (in place) with the rotation accumulated in
// S.Q[0]; at most `sweeps` sweeps, fewer when a sweep rotates nothing or no pair needs a rotation
// before a later sweep.  Each inner round: the
// first half-warp decides the 16 rotations; then every thread rotates one 2 x 2 block of G (rows
// of pair t / 16, columns of pair t % 16; the blocks partition G, so in place) and two column
// pairs of one row of Q.
__device__ __forceinline__ void bj_inner(BjShared& S, int sweeps, float tol, float noise) {
    const int tid = threadIdx.x;
    for (int e = tid; e < BJ_K * BJ_K; e += BJ_THREADS) S.Q[0][(e >> 5) * BJ_QLD + (e & 31)] = (e >> 5) == (e & 31);
    const int bi = tid >> 4, bj = tid & 15;          // G block
    const int qu = tid >> 3, qj = 2 * (tid & 7);      // Q row, first column pair
    float* Qr = S.Q[0] + qu * BJ_QLD;
    for (int isw = 0; isw < sweeps; ++isw) {
        if (isw > 0) {
            // a later sweep only if some pair still needs a rotation (one block-wide test instead
            // of 31 rounds of decisions; the outer test always holds before the first sweep)
            int need = 0;
            for (int e = tid; e < BJ_K * BJ_K; e += BJ_THREADS) {
                const int u = e >> 5, v = e & 31;
                if (u < v) need |= bj_need(S.G[u * BJ_LD + v], S.G[u * BJ_LD + u], S.G[v * BJ_LD + v], tol, noise);
            }
            if (!__syncthreads_or(need)) break;
        }
        int any_sweep = 0;
        for (int rnd = 0; rnd < BJ_K - 1; ++rnd) {
            if (tid < 32) {
                int rot = 0;
                if (tid < BJ_NP) {
                    const int p = S.lo[rnd][tid], q = S.hi[rnd][tid];
                    const float gpp = S.G[p * BJ_LD + p], gqq = S.G[q * BJ_LD + q], gpq = S.G[p * BJ_LD + q];
                    float c = 1.f, sn = 0.f;
                    if (bj_need(gpq, gpp, gqq, tol, noise)) {
                        bj_rot(gpp, gqq, gpq, c, sn);
                        rot = 1;
                    }
                    S.c[tid] = c;
                    S.s[tid] = sn;
                }
                const unsigned b = __ballot_sync(0xffffffffu, rot);
                if (tid == 0) S.flag[rnd & 1] = b != 0u;
            }
            __syncthreads();
            if (!S.flag[rnd & 1]) continue;   // nothing rotated: G and Q unchanged this round
            any_sweep = 1;
            {
                const int p0 = S.lo[rnd][bi], q0 = S.hi[rnd][bi], p1 = S.lo[rnd][bj], q1 = S.hi[rnd][bj];
                const float ci = S.c[bi], si = S.s[bi], cj = S.c[bj], sj = S.s[bj];
                float* G = S.G;
                const float a = G[p0 * BJ_LD + p1], b = G[p0 * BJ_LD + q1];
                const float c = G[q0 * BJ_LD + p1], d = G[q0 * BJ_LD + q1];
                // columns (p1, q1) by (cj, sj), then rows (p0, q0) by (ci, si)
                const float a1 = cj * a - sj * b, b1 = sj * a + cj * b;
                const float c1 = cj * c - sj * d, d1 = sj * c + cj * d;
                G[p0 * BJ_LD + p1] = ci * a1 - si * c1;
                G[q0 * BJ_LD + p1] = si * a1 + ci * c1;
                G[p0 * BJ_LD + q1] = ci * b1 - si * d1;
                G[q0 * BJ_LD + q1] = si * b1 + ci * d1;
            }
            {
                const int pa = S.lo[rnd][qj], qa = S.hi[rnd][qj];
                const int pb = S.lo[rnd][qj + 1], qb = S.hi[rnd][qj + 1];
                const float ca = S.c[qj], sa = S.s[qj], cb = S.c[qj + 1], sb = S.s[qj + 1];
                const float xa = Qr[pa], ya = Qr[qa], xb = Qr[pb], yb = Qr[qb];
                Qr[pa] = ca * xa - sa * ya;
                Qr[qa] = sa * xa + ca * ya;
                Qr[pb] = cb * xb - sb * yb;
                Qr[qb] = sb * xb + cb * yb;
            }
            __syncthreads();
        }
        if (!any_sweep) break;
    }
}

// V(:, gcol) <- V(:, gcol) Qp for the k columns gcol of V (ld rows, `rows` of them), straight from
// and to global memory: a thread takes whole rows (32 loads coalesced across the warp, the 32 x 32
// products from Qp in shared memory in two halves of 16 output columns, 32 stores).
__device__ __forceinline__ void bj_rotate_global(float* __restrict__ A, int ld, int rows, const float* __restrict__ Qp,
                                                 const int* __restrict__ gcol, int k) {
    for (int r = threadIdx.x; r < rows; r += BJ_THREADS) {
        float x[BJ_K];
#pragma unroll
        for (int u = 0; u < BJ_K; ++u) x[u] = (u < k) ? A[(long long)gcol[u] * ld + r] : 0.f;
#pragma unroll
        for (int h = 0; h < BJ_K; h += 16) {
            float acc[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) acc[j] = 0.f;
#pragma unroll
            for (int u = 0; u < BJ_K; ++u) {
#pragma unroll
                for (int j4 = 0; j4 < 16; j4 += 4) {
                    const float4 q = *reinterpret_cast<const float4*>(Qp + u * BJ_QLD + h + j4);
                    acc[j4] = fmaf(x[u], q.x, acc[j4]);
                    acc[j4 + 1] = fmaf(x[u], q.y, acc[j4 + 1]);
                    acc[j4 + 2] = fmaf(x[u], q.z, acc[j4 + 2]);
                    acc[j4 + 3] = fmaf(x[u], q.w, acc[j4 + 3]);
                }
            }
#pragma unroll
            for (int j = 0; j < 16; ++j)
                if (h + j < k) A[(long long)gcol[h + j] * ld + r] = acc[j];
        }
    }
}

// Rotate the k columns gcol of A (ld rows, `rows` of them) by Qp, staging at most `cap` rows at
// a time in X.
__device__ __forceinline__ void bj_rotate_streamed(float* __restrict__ X, float* __restrict__ A, int ld, int rows,
                                                   int cap, const float* __restrict__ Qp, const int* __restrict__ gcol,
                                                   int k) {
    for (int r0 = 0; r0 < rows; r0 += cap) {
        const int len = min(cap, rows - r0);
        bj_stage_async(X, A, ld, r0, len, gcol);
        cp_async_commit();
        cp_async_wait<0>();
        __syncthreads();
        bj_rotate(X, Qp, len);
        __syncthreads();
        bj_unstage(X, A, ld, r0, len, gcol, k);
        __syncthreads();
    }
}

// One block pair.  Returns (in every thread) the FP32 flops of its Gram matrix and, if it rotated,
// of the column rotations (negative when it rotated: -flops), 0 when the round has no task for
// it.  XW holds `cap` staged rows; XV
// (n rows) is a separate area when `split` (V then loads while W is processed), else it aliases
// XW.  A sector taller than cap is streamed through XW in row chunks (its W is read twice: once
// for the Gram matrix, once for the rotation).
__device__ double bj_task(BjShared& S, float* __restrict__ XW, float* __restrict__ XV, int cap, const SvdSec& s,
                        const BjSec& b, int si, int pi, int round, float* __restrict__ W, float* __restrict__ V,
                        float tol, float noise_c, float* __restrict__ gmax, int inner_sweeps,
                        int* __restrict__ bmod, int* __restrict__ pchk, int now) {
    int cI, kI, cJ, kJ, I = 0, J = 0;
    if (b.nb == 1) {
        if (round != 0) return 0.0;
        cI = 0; kI = s.n; cJ = 0; kJ = 0;
    } else {
        if (round >= b.nbp - 1) return 0.0;
        I = rr_pos(pi, round, b.nbp);
        J = rr_pos(b.nbp - 1 - pi, round, b.nbp);
        if (I > J) { const int t = I; I = J; J = t; }
        if (J >= b.nb) return 0.0;
        cI = I * BJ_B; kI = min(BJ_B, s.n - cI);
        cJ = J * BJ_B; kJ = min(BJ_B, s.n - cJ);
    }
    // skip a pair found converged after both blocks' last rotations (same values in every thread)
    int* const chk = pchk + b.pst0 + I * b.nb + J;
    if (__ldcg(chk) > max(__ldcg(bmod + b.blk0 + I), __ldcg(bmod + b.blk0 + J))) return 0.0;
    const int k = kI + kJ;
    const int tid = threadIdx.x;
    const double gram_flops = 2.0 * s.p * k * k, rot_flops = 2.0 * ((double)s.p + s.n) * k * k;
    const bool resident = s.p <= cap;                 // W's columns fit: staged once
    const bool split = resident && XV != XW;          // and V's alongside
    if (tid < BJ_K) S.gcol[tid] = tid < kI ? cI + tid : (tid < k ? cJ + tid - kI : -1);
    __syncthreads();
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
    if (resident) {
        bj_stage_async(XW, W + s.w_off, s.p, 0, s.p, S.gcol);
        cp_async_commit();
        if (split) bj_stage_async(XV, V + s.v_off, s.n, 0, s.n, S.gcol);
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        bj_gram_acc(acc, XW, s.p);
    } else {
        for (int r0 = 0; r0 < s.p; r0 += cap) {
            const int len = min(cap, s.p - r0);
            bj_stage_async(XW, W + s.w_off, s.p, r0, len, S.gcol);
            cp_async_commit();
            cp_async_wait<0>();
            __syncthreads();
            bj_gram_acc(acc, XW, len);
            __syncthreads();
        }
    }
    bj_gram_reduce(S, acc);
    __syncthreads();
    if (tid < 32) {
        float d = tid < k ? S.G[tid * BJ_LD + tid] : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) d = fmaxf(d, __shfl_xor_sync(0xffffffffu, d, o));
        if (tid == 0) {
            float g = *((volatile float*)&gmax[si]);
            if (d > g) {
                atomicMax(reinterpret_cast<int*>(&gmax[si]), __float_as_int(d));
                g = d;
            }
            S.noise = noise_c * sqrtf(g);
        }
    }
    __syncthreads();
    const float noise = S.noise;
    int need = 0;
    for (int e = tid; e < BJ_K * BJ_K; e += BJ_THREADS) {
        const int u = e >> 5, v = e & 31;
        if (u < v && v < k)
            need |= bj_need(S.G[u * BJ_LD + v], S.G[u * BJ_LD + u], S.G[v * BJ_LD + v], tol, noise);
    }
    if (!__syncthreads_or(need)) {
        cp_async_wait<0>();
        __syncthreads();
        if (tid == 0) *chk = now;
        return gram_flops;
    }
    bj_inner(S, inner_sweeps, tol, noise);
    const float* Gf = S.G;
    // order the eigenvectors of the k real columns by decreasing eigenvalue (ties: lower index
    // first); the padding columns are never rotated and keep their positions k..31 (a real
    // column of a numerically rank-deficient pair can end with an eigenvalue rounded below zero,
    // which must not trade places with a padding column's zero)
    if (tid < BJ_K) S.diag[tid] = Gf[tid * BJ_LD + tid];
    __syncthreads();
    if (tid < BJ_K) {
        const float d = S.diag[tid];
        int r = tid;
        if (tid < k) {
            r = 0;
            for (int v = 0; v < k; ++v) r += (S.diag[v] > d) || (S.diag[v] == d && v < tid);
        }
        S.perm[r] = tid;
    }
    __syncthreads();
    float* Qp = S.Q[1];
    for (int e = tid; e < BJ_K * BJ_K; e += BJ_THREADS) {
        const int u = e >> 5, r = e & 31;
        Qp[u * BJ_QLD + r] = S.Q[0][u * BJ_QLD + S.perm[r]];
    }
    __syncthreads();
    if (resident) {
        bj_rotate(XW, Qp, s.p);
        __syncthreads();
        bj_unstage(XW, W + s.w_off, s.p, 0, s.p, S.gcol, k);
        if (split) {
            cp_async_wait<0>();
            __syncthreads();
            bj_rotate(XV, Qp, s.n);
            __syncthreads();
            bj_unstage(XV, V + s.v_off, s.n, 0, s.n, S.gcol, k);
            __syncthreads();
            if (tid == 0) bmod[b.blk0 + I] = bmod[b.blk0 + J] = now;
            return -(gram_flops + rot_flops);
        }
        __syncthreads();
    } else {
        bj_rotate_streamed(XW, W + s.w_off, s.p, s.p, cap, Qp, S.gcol, k);
    }
    bj_rotate_global(V + s.v_off, s.n, s.n, Qp, S.gcol, k);
    __syncthreads();
    if (tid == 0) bmod[b.blk0 + I] = bmod[b.blk0 + J] = now;
    return -(gram_flops + rot_flops);
}

// One round of one sweep: every CTA takes tasks blockIdx.x, blockIdx.x + gridDim.x, ...
// rot[sweep] counts the pairs rotated in this sweep (zeroed by the host).  A launch whose previous
// sweep rotated nothing returns at once (the host enqueues a sweep before it has read the result
// of the one before).
__global__ void __launch_bounds__(BJ_THREADS, 1)
    k_bjacobi_round(const SvdSec* __restrict__ secs, const BjSec* __restrict__ bsecs, const int* __restrict__ task_sec,
                    int ntasks, int round, int sweep, int nrounds, int inner_sweeps, int max_p, int split,
                    float* __restrict__ W, float* __restrict__ V, float noise_c, float* __restrict__ gmax,
                    int* __restrict__ bmod, int* __restrict__ pchk, int* __restrict__ rot,
                    unsigned long long* __restrict__ flops) {
    extern __shared__ __align__(16) unsigned char bj_smem[];
    if (sweep > 0 && *((volatile int*)&rot[sweep - 1]) == 0) return;
    BjShared& S = *reinterpret_cast<BjShared*>(bj_smem);
    float* XW = reinterpret_cast<float*>(bj_smem + sizeof(BjShared));
    float* XV = split ? XW + (size_t)max_p * BJ_LD : XW;
    for (int e = threadIdx.x; e < (BJ_K - 1) * BJ_NP; e += blockDim.x) {
        const int rnd = e / BJ_NP, i = e % BJ_NP;
        const int a = rr_pos(i, rnd, BJ_K), b = rr_pos(BJ_K - 1 - i, rnd, BJ_K);
        S.lo[rnd][i] = (unsigned char)min(a, b);
        S.hi[rnd][i] = (unsigned char)max(a, b);
    }
    __syncthreads();
    double fl = 0.0;
    for (int t = blockIdx.x; t < ntasks; t += gridDim.x) {
        const int si = task_sec[t];
        const SvdSec s = secs[si];
        const BjSec b = bsecs[si];
        const double r = bj_task(S, XW, XV, max_p, s, b, si, t - b.task0, round, W, V, b.tol, noise_c, gmax,
                                 inner_sweeps, bmod, pchk, sweep * nrounds + round + 1);
        fl += fabs(r);
        if (r < 0.0 && threadIdx.x == 0) atomicAdd(&rot[sweep], 1);
    }
    if (threadIdx.x == 0 && fl > 0.0) atomicAdd(flops, (unsigned long long)fl);
}

// All sweeps in one cooperative launch, for a caller that has the GPU to itself, without grid-wide
// barriers.  Work items (sweep, round, sector, pair) are taken in order from one counter: per sweep
// the rounds in order, in each round every sector's pairs (taller sectors first).  An item waits
// only for the previous round of its own sector (the sector's count of finished items), since
// sectors are independent: the small sectors run ahead into later sweeps while the tall sectors'
// long round sequences are in flight, instead of every round of every sector waiting for the
// slowest pair of the whole batch.  Items depend on earlier items only and every CTA is resident,
// so the queue always drains.  A sector whose sweep rotated nothing has converged: its later items
// are counted without work, and the launch ends once every sector has converged (or after
// max_sweeps; nact = sectors with columns).  A dependency wait is bounded (ERRBIT_TIMEOUT and the
// abort flag after 2 s).
// qstate (zeroed): [0] next item, [1] converged sectors, [2] abort flag, then finished items per
// sector (nsec), converged flags (nsec), pairs rotated per sector and sweep (nsec x max_sweeps).
// rot[sweep]: pairs rotated in that sweep over all sectors; *sweeps: sweeps run by the slowest
// sector.
__global__ void __launch_bounds__(BJ_THREADS, 1)
    k_bjacobi_queue(const SvdSec* __restrict__ secs, const BjSec* __restrict__ bsecs, const int2* __restrict__ items,
                    int per_sweep, int nsec, int nact, int nrounds, int max_sweeps, int inner_sweeps, int max_p,
                    int split,
                    float* __restrict__ W, float* __restrict__ V, float noise_c, float* __restrict__ gmax,
                    int* __restrict__ bmod, int* __restrict__ pchk, int* __restrict__ qstate, int* __restrict__ rot,
                    int* __restrict__ sweeps, unsigned* __restrict__ err, unsigned long long* __restrict__ flops) {
    extern __shared__ __align__(16) unsigned char bj_smem[];
    BjShared& S = *reinterpret_cast<BjShared*>(bj_smem);
    float* XW = reinterpret_cast<float*>(bj_smem + sizeof(BjShared));
    float* XV = split ? XW + (size_t)max_p * BJ_LD : XW;
    const int tid = threadIdx.x;
    for (int e = tid; e < (BJ_K - 1) * BJ_NP; e += blockDim.x) {
        const int rnd = e / BJ_NP, i = e % BJ_NP;
        const int a = rr_pos(i, rnd, BJ_K), b = rr_pos(BJ_K - 1 - i, rnd, BJ_K);
        S.lo[rnd][i] = (unsigned char)min(a, b);
        S.hi[rnd][i] = (unsigned char)max(a, b);
    }
    int* const qnext = qstate;
    int* const nconv = qstate + 1;
    int* const abort_flag = qstate + 2;
    int* const done = qstate + 3;
    int* const conv = done + nsec;
    int* const srot = conv + nsec;
    const long long total = (long long)per_sweep * max_sweeps;
    double fl = 0.0;
    for (;;) {
        if (tid == 0) S.qitem = atomicAdd(qnext, 1);
        __syncthreads();
        const long long i = S.qitem;
        if (i >= total) break;                       // uniform: read before anyone writes it again
        const int sweep = (int)(i / per_sweep);
        const int2 it = items[i - (long long)sweep * per_sweep];
        const int si = it.x, round = it.y >> 16, pi = it.y & 0xffff;
        const BjSec b = bsecs[si];
        const int nr = b.nb == 1 ? 1 : b.nbp - 1;
        if (tid == 0) {
            int state = 1;                           // 1: work, 0: count only, -1: count and leave
            if (*((volatile int*)abort_flag) != 0 || *((volatile int*)nconv) >= nact) state = -1;
            else if (*((volatile int*)&conv[si]) != 0) state = 0;
            if (state == 1) {
                const int need = (sweep * nr + round) * b.ntask;
                uint64_t t0;
                asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
                while (*((volatile int*)&done[si]) < need) {
                    if (*((volatile int*)abort_flag) != 0) { state = -1; break; }
                    uint64_t t;
                    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
                    if (t - t0 > 2000000000ull) {
                        atomicOr(err, ERRBIT_TIMEOUT);
                        atomicExch(abort_flag, 1);
                        state = -1;
                        break;
                    }
                }
                // the sector's earlier rounds (columns, stamps) happen before this item's loads
                __threadfence();
            }
            S.qok = state;
        }
        __syncthreads();
        const int state = S.qok;
        if (state == 1) {
            const SvdSec s = secs[si];
            const double r = bj_task(S, XW, XV, max_p, s, b, si, pi, round, W, V, b.tol, noise_c, gmax,
                                     inner_sweeps, bmod, pchk, sweep * nrounds + round + 1);
            fl += fabs(r);
            if (r < 0.0 && tid == 0) {
                atomicAdd(&srot[si * max_sweeps + sweep], 1);
                atomicAdd(&rot[sweep], 1);
            }
        }
        __syncthreads();                             // every thread's writes precede the count
        if (tid == 0) {
            __threadfence();
            const int old = atomicAdd(&done[si], 1);
            if (old + 1 == (sweep + 1) * nr * b.ntask) {   // the last item of this sector's sweep
                __threadfence();
                if (*((volatile int*)&conv[si]) == 0) {
                    atomicMax(sweeps, sweep + 1);
                    if (*((volatile int*)&srot[si * max_sweeps + sweep]) == 0) {
                        atomicExch(&conv[si], 1);
                        atomicAdd(nconv, 1);
                    }
                }
            }
        }
        if (state < 0) break;
    }
    if (tid == 0 && fl > 0.0) atomicAdd(flops, (unsigned long long)fl);
}

}  // namespace

int bjacobi_max_rows() { return (int)((BJ_SMEM_MAX - sizeof(BjShared)) / (BJ_LD * sizeof(float))); }

void launch_bjacobi(const SvdSec* secs, const BjSec* bsecs, const int* task_sec, int ntasks, int nrounds, int max_rows,
                    int max_n, int max_sweeps, int inner_sweeps, float* W, float* V, float noise_c,
                    float* gmax, int* bmod, int* pchk, int* rot, int* sweeps, unsigned* bar, unsigned* err,
                    unsigned long long* flops, const int2* items, int per_sweep, int nsec, int nact, int* qstate,
                    cudaStream_t st) {
    if (ntasks <= 0 || nrounds <= 0) {
        PD_CK(cudaMemsetAsync(sweeps, 0, sizeof(int), st));
        return;
    }
    // taller sectors are streamed through the staging area in chunks of max_rows rows
    max_rows = std::max(1, std::min(max_rows, bjacobi_max_rows()));
    // W and V staged side by side when both fit (V then loads while W is processed)
    const size_t row_bytes = BJ_LD * sizeof(float);
    int split = sizeof(BjShared) + (size_t)(max_rows + max_n) * row_bytes <= (size_t)BJ_SMEM_MAX;
    const size_t smem = sizeof(BjShared) + (size_t)(split ? max_rows + max_n : max_rows) * row_bytes;
    // the shared-memory ceiling is raised once per process to the largest size any launch uses
    // (region threads launch concurrently with different sizes)
    static const cudaError_t attr =
        cudaFuncSetAttribute(k_bjacobi_round, cudaFuncAttributeMaxDynamicSharedMemorySize, BJ_SMEM_MAX);
    PD_CK(attr);
    int dev = 0, sms = 0;
    PD_CK(cudaGetDevice(&dev));
    PD_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (g_sm_cap == 0) {
        // the GPU is this caller's: all sweeps in one cooperative launch (the dependency queue)
        static const cudaError_t attr_c =
            cudaFuncSetAttribute(k_bjacobi_queue, cudaFuncAttributeMaxDynamicSharedMemorySize, BJ_SMEM_MAX);
        PD_CK(attr_c);
        int per_sm = 0;
        PD_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bjacobi_queue, BJ_THREADS, smem));
        PD_REQUIRE(per_sm > 0, DMRG_ERR_CAPACITY, "block Jacobi: kernel does not fit on an SM");
        const int cblocks = std::max(1, std::min(per_sweep, per_sm * sms));
        PD_CK(cudaMemsetAsync(sweeps, 0, sizeof(int), st));
        void* args[] = {(void*)&secs, (void*)&bsecs, (void*)&items, (void*)&per_sweep, (void*)&nsec, (void*)&nact,
                        (void*)&nrounds,
                        (void*)&max_sweeps, (void*)&inner_sweeps, (void*)&max_rows, (void*)&split, (void*)&W,
                        (void*)&V, (void*)&noise_c, (void*)&gmax, (void*)&bmod, (void*)&pchk, (void*)&qstate,
                        (void*)&rot, (void*)&sweeps, (void*)&err, (void*)&flops};
        PD_CK(cudaLaunchCooperativeKernel((void*)k_bjacobi_queue, cblocks, BJ_THREADS, args, smem, st));
        PD_LAUNCHED();
        return;
    }
    // regions run concurrently: one launch per round, nothing spins
    const int blocks = std::max(1, std::min(ntasks, 4 * sms));
    // rounds are enqueued sweep by sweep; the host reads rot of sweep s - 1 after enqueuing sweep s
    // (pinned copy + event), so the device never waits for the host; a sweep enqueued after the
    // converged one returns at once.
    int* hrot = sweep_flags_host(max_sweeps);
    std::vector<cudaEvent_t> evs(max_sweeps, nullptr);
    int done = max_sweeps;
    try {
        for (int sweep = 0; sweep < max_sweeps; ++sweep) {
            for (int round = 0; round < nrounds; ++round) {
                k_bjacobi_round<<<blocks, BJ_THREADS, smem, st>>>(secs, bsecs, task_sec, ntasks, round, sweep,
                                                                   nrounds, inner_sweeps, max_rows, split, W, V,
                                                                   noise_c, gmax, bmod, pchk, rot, flops);
                PD_LAUNCHED();
            }
            PD_CK(cudaMemcpyAsync(hrot + sweep, rot + sweep, sizeof(int), cudaMemcpyDeviceToHost, st));
            PD_CK(cudaEventCreateWithFlags(&evs[sweep], cudaEventDisableTiming));
            PD_CK(cudaEventRecord(evs[sweep], st));
            if (sweep > 0) {
                PD_CK(cudaEventSynchronize(evs[sweep - 1]));
                if (hrot[sweep - 1] == 0) {
                    done = sweep;      // sweep - 1 rotated nothing; the launches of `sweep` exit at once
                    break;
                }
            }
        }
        if (done == max_sweeps) {
            PD_CK(cudaEventSynchronize(evs[max_sweeps - 1]));
            if (hrot[max_sweeps - 1] == 0) done = max_sweeps;
        }
    } catch (...) {
        for (auto e : evs)
            if (e) cudaEventDestroy(e);
        throw;
    }
    for (auto e : evs)
        if (e) cudaEventDestroy(e);
    PD_CK(cudaMemcpyAsync(sweeps, &done, sizeof(int), cudaMemcpyHostToDevice, st));
}

}  // namespace pd
