// Internal declarations of the pdmrg engine (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <algorithm>
#include <atomic>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/pdmrg.h"

namespace pd {

// ------------------------------------------------------------------------------------------
// Errors
// ------------------------------------------------------------------------------------------
struct Error {
    dmrg_status st;
    std::string msg;
};

#define PD_CK(x)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (x);                                                             \
        if (e_ != cudaSuccess)                                                            \
            throw ::pd::Error{e_ == cudaErrorMemoryAllocation ? DMRG_ERR_OOM : DMRG_ERR_CUDA, \
                              std::string(#x) + ": " + cudaGetErrorString(e_)};            \
    } while (0)

#define PD_REQUIRE(cond, code, what)                                                      \
    do {                                                                                  \
        if (!(cond)) throw ::pd::Error{code, what};                                       \
    } while (0)

// Kernel launches issued by the library (process-wide counter).
extern std::atomic<long long> g_launches;
#define PD_LAUNCHED()                                                   \
    do {                                                                \
        PD_CK(cudaGetLastError());                                      \
        ::pd::g_launches.fetch_add(1, std::memory_order_relaxed);       \
    } while (0)

// Profiling classes of grouped-GEMM launches; the class of tensor-core launches comes from the
// calling thread's current activity.
enum ProfClass { PROF_MV = 0, PROF_ENV = 1, PROF_F64 = 2, PROF_F32 = 3, PROF_NONE = 4 };   // NONE: not tallied
extern thread_local int g_prof_class;
bool prof_on();
// With profiling on: record an event pair around a launch (call prof_start before the launch,
// prof_stop after); the elapsed time is resolved in dmrg_profile_read.
void* prof_start(cudaStream_t st);
void prof_stop(void* token, cudaStream_t st, int cls, double flops);
// Jacobi SVD statistics (sweeps run per call), accumulated while profiling is on; kind 0: FP32
// scalar Jacobi, 1: FP32 block Jacobi, 2: FP64; max_rows: the call's largest sector row count;
// flops: the FP32 Gram and rotation flops of a block-Jacobi call; rot_hist: its rotations per sweep.
void prof_svd(int sweeps, double ms, int kind, int max_rows, double flops, const int* rot_hist, int nhist,
              int bonds = 1, double alg_flops = 0.0, double alg_bytes = 0.0);
// An FP32 split redone in FP64 (counted always, not only while profiling).
void prof_fallback();
// An emulated FP64 GEMM batch sent to the FP64 units by its scale guard (counted always).
void prof_emu_fallback();

// Persistent and cooperative grids are sized to the SMs of the device; while R regions run
// concurrently (one host thread each), each thread caps its grids at sms / R so that the regions
// share the GPU spatially instead of queueing behind each other's resident grids.
extern thread_local int g_sm_cap;   // 0: no cap
inline int sm_share(int sms) { return g_sm_cap > 0 ? std::max(1, std::min(sms, g_sm_cap)) : sms; }

// Pinned host words (one per sweep, at least n) owned by the calling thread, for reading the
// per-sweep rotation flags of the Jacobi kernels without a device-wide synchronisation.
int* sweep_flags_host(int n);

// Device error word bits (written by kernels, read by the host after a step).
enum : unsigned {
    ERRBIT_TIMEOUT = 1u,      // a bounded mbarrier wait ran out
    ERRBIT_NONFINITE = 2u,    // NaN/Inf seen in a checked vector
    ERRBIT_BOUNDS = 4u,       // an index check failed (access skipped)
};

// ------------------------------------------------------------------------------------------
// Grouped GEMM contract shared by the FP64 SIMT engine and the tcgen05 engine:
//   C(m, n) (+)= alpha * sum_segments sum_k A(m, k) B(n, k)
//   A(m, k) = A[a_off + m*sam + k*sak], B(n, k) = B[b_off + n*sbn + k*sbk],
//   C(m, n) = C[c_off + m*scm + n*scn].
// The tensor-core engine requires sak = sbk = scm = 1, a uniform sam (= lda) per launch for A
// and sbn (= ldb) for B, and zero padding of every operand row up to the K tile.
// ------------------------------------------------------------------------------------------
struct GSeg {
    long long a_off, b_off;
    int K;
    int pad_;
};
struct GProb {
    int M, N;
    int seg0, nseg;
    long long c_off;
    int sam, sak, sbn, sbk, scm, scn;
    int accumulate;       // 0: C = alpha*AB, 1: C += alpha*AB
    int pad_;
    double alpha;
};
struct GTile {
    int prob, m0, n0, pad_;
};

// Block copy job: dst[r*drs + c*dcs] = scale * src[r*srs + c*scs] for r < rows, c < cols;
// zero columns cols <= c < zero_to (row-major destination only, dcs = 1).
struct CopyJob {
    long long src, dst;
    int rows, cols;
    int srs, scs, drs, dcs;
    int zero_to;
    int pad_;
    double scale;
};

// Linear combination of blocks: out[r*ldo + c] = sum_t coef_t * in[src_t + r*ld_t + c],
// zero-filled for cols <= c < zero_to.
struct MixJob {
    long long dst;
    int rows, cols, ldo, zero_to;
    int t0, nt;
};
struct MixTerm {
    long long src;
    int ld, pad_;
    double coef;
};

// Diagonal of H_eff: out[off + a*cols + c] = sum_t coef_t * Ld_t[a] * Rd_t[c], where
// Ld_t[a] = Lslab[l_t + a*(ldl+1)], Rd_t[c] = Rslab[r_t + c*(ldr+1)].
struct DiagJob {
    long long off;
    int rows, cols, t0, nt;
};
struct DiagTerm {
    long long l, r;
    double coef;
};

// ------------------------------------------------------------------------------------------
// Launch wrappers (kernels.cu)
// ------------------------------------------------------------------------------------------
template <class T>
void launch_gemm_simt(const GProb* probs, const GSeg* segs, const GTile* tiles, int ntiles, const T* A, const T* B,
                      T* C, cudaStream_t st);

// Elementwise block kernels run one CTA per chunk of CHUNK elements of one job; `chunks`
// lists (job, first element) for every chunk (built on the host, see make_chunks).
constexpr int CHUNK = 2048;
template <class Tin, class Tout>
void launch_copy(const CopyJob* jobs, const int2* chunks, int nchunks, const Tin* src, Tout* dst,
                 cudaStream_t st);

template <class Tin, class Tout>
void launch_mix(const MixJob* jobs, const int2* chunks, int nchunks, const MixTerm* terms,
                const Tin* in, Tout* out, cudaStream_t st);

template <class T>
void launch_diag(const DiagJob* jobs, const int2* chunks, int nchunks, const DiagTerm* terms,
                 const T* Lslab, int ldl, const T* Rslab, int ldr, double* out, cudaStream_t st);

// Chunk table for jobs of the given element counts.
inline std::vector<int2> make_chunks(const std::vector<long long>& elems) {
    std::vector<int2> c;
    for (size_t j = 0; j < elems.size(); ++j)
        for (long long e = 0; e < elems[j]; e += CHUNK) c.push_back(make_int2((int)j, (int)e));
    return c;
}

// Davidson helpers (all FP64, vectors of length n, basis rows of stride ldv)
void launch_dots(const double* V, long long ldv, int k, const double* y, long long n,
                 double* partial, int nchunks, double* out, cudaStream_t st);
void launch_ritz(const double* V, const double* AV, long long ldv, int k, const double* yth,
                 long long n, double* u, double* Au, double* r, double* partial, int nchunks,
                 double* norms, cudaStream_t st);
void launch_precond(const double* r, const double* diag, const double* theta, double floor_,
                    long long n, double* t, cudaStream_t st);
void launch_subtract(const double* V, long long ldv, int k, const double* c, long long n,
                     double* t, cudaStream_t st);
void launch_scale(const double* x, const double* nrm2, long long n, double* y, int invert_sqrt,
                  cudaStream_t st);
void launch_small_eig(const double* G, int k, int ldg, double* yth, cudaStream_t st);
void launch_nrm2(const double* x, long long n, double* partial, int nchunks, double* out,
                 cudaStream_t st);
void launch_finite_check(const double* x, long long n, unsigned* err, cudaStream_t st);

// One-sided Jacobi SVD over a batch of column-major matrices W_s (p_s x n_s, n_s <= p_s)
struct SvdSec {
    long long w_off;      // W: p x n column-major
    long long v_off;      // V: n x n column-major
    long long s_off;      // singular values / order buffers (n entries)
    int p, n;
    int npad;             // n rounded up to even
    int pair0;            // first global pair index of this sector in a round
};
template <class T>
void launch_svd_init_v(const SvdSec* secs, int nsec, int max_n, T* V, cudaStream_t st);
// All Jacobi sweeps (until a sweep without rotation, at most max_sweeps) in one cooperative launch.
// A pair of columns with Gram entries a, b, g is rotated when |g| > tol sqrt(p) sqrt(a b), p the
// row count of its own sector (the rounding noise of a p-long dot product grows like sqrt(p)).
// Pairs whose smaller column norm is below eta * |W_sector|_F are not rotated (eta = 0: all are).
// floor2: nsec doubles of scratch (unused when eta = 0).
// bar: 3 unsigned words of scratch for the bounded grid barrier; err: device error word.
template <class T>
void launch_jacobi(const SvdSec* secs, int nsec, const int* pair_sec, int npairs, int maxnpad, int max_sweeps, T* W,
                   T* V, T tol, double eta, double* floor2, int* rot, int* sweeps, unsigned* bar, unsigned* err,
                   cudaStream_t st);
// Block one-sided Jacobi (FP32, blocks of 16 columns) over the same sector batch.  Per sector:
// nb = ceil(n / 16) blocks, nbp = nb rounded up to even, task0 = first task of the sector in a
// round, ntask = tasks per round (nbp / 2; 1 when nb = 1).  task_sec[t] = sector of task t.
// tol: the sector's relative rotation threshold (FP32 dot products of p-long columns carry about
// eps * sqrt(p) relative noise, so it sits above that).  blk0 / pst0: the sector's first entry in
// the block and pair stamp arrays (nb and nb * nb entries).
struct BjSec {
    int nb, nbp, task0, ntask;
    float tol;
    int blk0, pst0;
};
int bjacobi_max_rows();
void launch_bjacobi(const SvdSec* secs, const BjSec* bsecs, const int* task_sec, int ntasks, int nrounds, int max_rows,
                    int max_n, int max_sweeps, int inner_sweeps, float* W, float* V, float noise_c, float* gmax,
                    int* bmod, int* pchk, int* rot, int* sweeps, unsigned* bar, unsigned* err,
                    unsigned long long* flops, const int2* items, int per_sweep, int nsec, int nact, int* qstate,
                    cudaStream_t st);
template <class T>
void launch_svd_finish(const SvdSec* secs, int nsec, const T* W, double* sig, int* order, cudaStream_t st);

// Truncation selection over all sectors.  sig sorted per sector by `order`; sectors packed
// back to back (s_off = prefix sums).  Scratch: (total + nsec) doubles, 3*total ints.
void launch_truncate(const SvdSec* secs, int nsec, const double* sig, const int* order, int total, int m_max,
                     double rel_cutoff, double degen_tol, int* kept, double* weights, double* scratch_d, int* scratch_i,
                     cudaStream_t st);

}  // namespace pd
