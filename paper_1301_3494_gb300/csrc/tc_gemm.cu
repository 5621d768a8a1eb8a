// tcgen05 grouped GEMM for sm_103a: BF16 (kind::f16) or TF32 (kind::tf32) operands, FP32
// accumulation in tensor memory.  Serves the block contractions of the projected Hamiltonian
// (L stage and R stage) and of the projected-operator updates (Sec. II) in mixed precision.
//
// Contract (see internal.h): C(m, n) (+)= alpha * sum_seg sum_k A[a_off + m*lda + k] B[b_off + n*ldb + k],
// stored at C[c_off + m + n*ldc].  A and B are row slabs with a uniform leading dimension, rows
// zero-padded to a multiple of 64 elements, so every k-block is a full 128-byte TMA box.
//
// Kernel: persistent, one CTA per SM, 6 warps:
//   warp 0      TMA producer (one lane): 2D tiled loads, SWIZZLE_128B, S-stage mbarrier ring
//   warp 1      TMEM owner + MMA issuer (one lane): tcgen05.mma 128 x BN x (32 bytes of K)
//   warps 2..5  epilogue: tcgen05.ld 32x32b from the accumulator, coalesced stores along m
// Two accumulators of BN columns each in TMEM, so the epilogue of tile i overlaps tile i+1.
// Every mbarrier wait is bounded by %globaltimer; on expiry the kernel sets ERRBIT_TIMEOUT,
// drains its own asynchronous work with bounded waits, frees TMEM and returns.
#include <cuda.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>

#include "plans.h"

namespace pd {

namespace {

constexpr int BM = 128;
constexpr int THREADS = 192;
constexpr uint64_t WAIT_NS = 2000000000ull;      // 2 s per wait before giving up
constexpr uint64_t DRAIN_NS = 500000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t a) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait.  Returns false if the CTA is aborting or the wait timed out (then aborts).
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, volatile int* abort_flag, unsigned* err) {
    if (mbar_try(a, parity)) return true;
    const uint64_t t0 = gtimer();
    for (uint32_t i = 0;; ++i) {
        if (mbar_try(a, parity)) return true;
        if ((i & 63) == 63) {
            if (*abort_flag) return false;
            if (gtimer() - t0 > WAIT_NS) {
                *abort_flag = 1;
                atomicOr(err, ERRBIT_TIMEOUT);
                return false;
            }
        }
    }
}
__device__ __forceinline__ bool mbar_wait_plain(uint32_t a, uint32_t parity, uint64_t ns) {
    const uint64_t t0 = gtimer();
    while (!mbar_try(a, parity))
        if (gtimer() - t0 > ns) return false;
    return true;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

template <int KIND>
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    if constexpr (KIND == 0) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc)
            : "memory");
    }
}

__device__ __forceinline__ void tc_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row atoms 1024 bytes apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1u << 16;                  // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024u >> 4) << 32;        // stride byte offset: next 8-row atom
    d |= (uint64_t)1u << 46;                  // descriptor version
    d |= (uint64_t)2u << 61;                  // SWIZZLE_128B
    return d;
}

// Instruction descriptor: FP32 accumulator, A/B format (1 = BF16, 2 = TF32), K-major A and B.
__host__ __device__ constexpr uint32_t make_idesc(int kind, int M, int N) {
    return (1u << 4) | ((kind == 0 ? 1u : 2u) << 7) | ((kind == 0 ? 1u : 2u) << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

template <int KIND, int BN, int STAGES, class OutT>
__global__ void __launch_bounds__(THREADS, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
              const GProb* __restrict__ probs, const GSeg* __restrict__ segs, const GTile* __restrict__ tiles,
              int ntiles, int lda, int ldb, OutT* __restrict__ C, unsigned* __restrict__ err) {
    constexpr int ESIZE = KIND == 0 ? 2 : 4;
    constexpr int BK = 128 / ESIZE;            // elements of K per stage (one 128-byte row)
    constexpr int A_BYTES = BM * 128;
    constexpr int B_BYTES = BN * 128;
    constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    constexpr int KSTEPS = 4;                   // 4 MMAs of 32 bytes of K each
    constexpr uint32_t IDESC = make_idesc(KIND, BM, BN);
    constexpr uint32_t TMEM_COLS = 2 * BN < 32 ? 32 : 2 * BN;

    extern __shared__ __align__(1024) unsigned char dsmem[];
    __shared__ __align__(8) uint64_t bar_full[STAGES], bar_empty[STAGES], bar_tfull[2], bar_tempty[2], bar_drain;
    __shared__ uint32_t tmem_base_s;
    __shared__ volatile int abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(dsmem) + 1023) & ~uintptr_t(1023));
    const uint32_t sbase = smem_u32(base);

    if (threadIdx.x == 0) {
        abort_flag = 0;
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(smem_u32(&bar_full[s]), 1);
            mbar_init(smem_u32(&bar_empty[s]), 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(smem_u32(&bar_tfull[s]), 1);
            mbar_init(smem_u32(&bar_tempty[s]), 4);
        }
        mbar_init(smem_u32(&bar_drain), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_s)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_s;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer ----------------
            int stage = 0;
            uint32_t phase = 0;
            int issued[STAGES];
            uint32_t issued_phase[STAGES];
            for (int s = 0; s < STAGES; ++s) issued[s] = 0, issued_phase[s] = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                const GTile tl = tiles[t];
                const GProb p = probs[tl.prob];
                for (int sgi = 0; sgi < p.nseg && ok; ++sgi) {
                    const GSeg sg = segs[p.seg0 + sgi];
                    const int ya = (int)(sg.a_off / lda) + tl.m0;
                    const int yb = (int)(sg.b_off / ldb) + tl.n0;
                    const int nkb = (sg.K + BK - 1) / BK;
                    for (int kb = 0; kb < nkb; ++kb) {
                        if (!mbar_wait(smem_u32(&bar_empty[stage]), phase ^ 1u, &abort_flag, err)) { ok = false; break; }
                        const uint32_t fb = smem_u32(&bar_full[stage]);
                        mbar_expect_tx(fb, STAGE_BYTES);
                        const uint32_t sa = sbase + stage * STAGE_BYTES;
                        tma_load_2d(sa, &tmA, kb * BK, ya, fb);
                        tma_load_2d(sa + A_BYTES, &tmB, kb * BK, yb, fb);
                        issued[stage] = 1;
                        issued_phase[stage] = phase;
                        if (++stage == STAGES) { stage = 0; phase ^= 1u; }
                    }
                }
            }
            if (!ok) {
                // drain: wait (bounded) until every load this thread issued has landed
                for (int s = 0; s < STAGES; ++s)
                    if (issued[s]) mbar_wait_plain(smem_u32(&bar_full[s]), issued_phase[s], DRAIN_NS);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            int stage = 0;
            uint32_t phase = 0;
            int acc = 0;
            uint32_t acc_phase = 0;
            bool ok = true, any = false;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                const GTile tl = tiles[t];
                const GProb p = probs[tl.prob];
                if (!mbar_wait(smem_u32(&bar_tempty[acc]), acc_phase ^ 1u, &abort_flag, err)) { ok = false; break; }
                tc_fence_after();
                const uint32_t dt = tmem + (uint32_t)(acc * BN);
                uint32_t accumulate = 0;
                for (int sgi = 0; sgi < p.nseg && ok; ++sgi) {
                    const GSeg sg = segs[p.seg0 + sgi];
                    const int nkb = (sg.K + BK - 1) / BK;
                    for (int kb = 0; kb < nkb; ++kb) {
                        if (!mbar_wait(smem_u32(&bar_full[stage]), phase, &abort_flag, err)) { ok = false; break; }
                        tc_fence_after();
                        const uint32_t sa = sbase + stage * STAGE_BYTES;
                        const uint32_t sb = sa + A_BYTES;
#pragma unroll
                        for (int k = 0; k < KSTEPS; ++k) {
                            tc_mma<KIND>(dt, sdesc(sa + 32 * k), sdesc(sb + 32 * k), IDESC, accumulate);
                            accumulate = 1;
                        }
                        tc_commit(smem_u32(&bar_empty[stage]));
                        any = true;
                        if (++stage == STAGES) { stage = 0; phase ^= 1u; }
                    }
                }
                if (!ok) break;
                tc_commit(smem_u32(&bar_tfull[acc]));
                if (++acc == 2) { acc = 0; acc_phase ^= 1u; }
            }
            if (!ok && any) {
                // drain: all MMAs issued so far complete before TMEM is released
                tc_commit(smem_u32(&bar_drain));
                mbar_wait_plain(smem_u32(&bar_drain), 0, DRAIN_NS);
            }
        }
    } else {
        // ---------------- epilogue (warps 2..5) ----------------
        const int quarter = warp & 3;
        int acc = 0;
        uint32_t acc_phase = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
            const GTile tl = tiles[t];
            const GProb p = probs[tl.prob];
            const bool ok = mbar_wait(smem_u32(&bar_tfull[acc]), acc_phase, &abort_flag, err);
            if (!__all_sync(0xffffffffu, ok)) break;
            tc_fence_after();
            const int m = tl.m0 + quarter * 32 + lane;
            const uint32_t trow = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(acc * BN);
            const int ncols = min(BN, p.N - tl.n0);
            // FP32 arithmetic only (FP64 issue rate is low on this part); one conversion for FP64 output
            const float alpha = (float)p.alpha;
            const bool scale = alpha != 1.0f;
            const bool accum = p.accumulate != 0;
            OutT* crow = C + p.c_off + (long long)m * p.scm;
            const int nlim = p.N - tl.n0;
            for (int c0 = 0; c0 < ncols; c0 += 32) {
                uint32_t r[32];
                tc_ld32(trow + (uint32_t)c0, r);
                if (m < p.M) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int n = c0 + j;
                        if (n < nlim) {
                            OutT* dst = crow + (long long)(tl.n0 + n) * p.scn;
                            float v = __uint_as_float(r[j]);
                            if (scale) v *= alpha;
                            if constexpr (std::is_same<OutT, double>::value) {
                                *dst = accum ? *dst + (double)v : (double)v;
                            } else {
                                if (accum) v += (float)*dst;
                                *dst = (OutT)v;
                            }
                        }
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&bar_tempty[acc]));
            if (++acc == 2) { acc = 0; acc_phase ^= 1u; }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// ------------------------------------------------------------------------------------------
// Host side
// ------------------------------------------------------------------------------------------
typedef CUresult (*EncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                             const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                             CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encode_fn() {
    static EncodeFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, []() {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeFn>(p);
    });
    return fn;
}

CUtensorMap make_map(Num t, const void* base, long long rows, int ld, int box_rows) {
    EncodeFn fn = encode_fn();
    PD_REQUIRE(fn != nullptr, DMRG_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
    PD_REQUIRE((reinterpret_cast<uintptr_t>(base) & 15) == 0, DMRG_ERR_ARG, "TMA base not 16-byte aligned");
    const int es = (int)num_size(t);
    PD_REQUIRE(((long long)ld * es) % 16 == 0, DMRG_ERR_ARG, "TMA row stride not a multiple of 16 bytes");
    CUtensorMap m;
    cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)std::max<long long>(rows, 1)};
    cuuint64_t strides[1] = {(cuuint64_t)ld * es};
    cuuint32_t box[2] = {(cuuint32_t)(128 / es), (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(&m, t == Num::BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                    const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    PD_REQUIRE(r == CUDA_SUCCESS, DMRG_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    return m;
}

int sm_count() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        PD_CK(cudaGetDevice(&dev));
        PD_CK(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
    }
    return n;
}

template <int KIND, int BN, int STAGES, class OutT>
void launch_tc(GemmBatch& g, const CUtensorMap& ma, const CUtensorMap& mb, int lda, int ldb, void* C, unsigned* err,
               cudaStream_t st) {
    constexpr int STAGE_BYTES = BM * 128 + BN * 128;
    constexpr int SMEM = STAGES * STAGE_BYTES + 1024;
    auto kern = k_tc_gemm<KIND, BN, STAGES, OutT>;
    static const cudaError_t attr = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
    PD_CK(attr);
    int grid = std::min(g.ntiles, sm_share(sm_count()));
    void* tok = prof_on() ? prof_start(st) : nullptr;
    kern<<<grid, THREADS, SMEM, st>>>(ma, mb, g.dprobs.as<GProb>(), g.dsegs.as<GSeg>(), g.dtiles.as<GTile>(), g.ntiles,
                                      lda, ldb, (OutT*)C, err);
    PD_LAUNCHED();
    if (tok) prof_stop(tok, st, g_prof_class, g.flops);
}

// Tile width from a cost model of the batch: padded MMA work at the tensor rate plus the
// operand bytes every tile streams through shared memory (A: 128 rows, B: BN rows per k-block)
// at an L2-to-SM rate.  Narrow tiles waste less padding on small blocks, wide tiles re-read
// A less often.
int pick_bn(const GemmBatch& g, int esize) {
    const double flop_rate = 2.0e15, byte_rate = 2.0e13;
    double best = -1.0;
    int bn_best = 128;
    for (int bn : {256, 128, 64}) {
        double t = 0.0;
        for (const auto& p : g.probs) {
            long long kpad = 0;
            for (int s = 0; s < p.nseg; ++s) kpad += (long long)((g.segs[p.seg0 + s].K + 63) / 64) * 64;
            const double tiles = (double)((p.M + BM - 1) / BM) * ((p.N + bn - 1) / bn);
            t += tiles * (2.0 * BM * bn * kpad / flop_rate + (double)kpad * (BM + bn) * esize / byte_rate);
        }
        if (best < 0 || t < best) { best = t; bn_best = bn; }
    }
    return bn_best;
}

// Measured tile-width autotuner.  A batch's shape class (operand and output types, and the
// rounded logarithms of its flops (in pairs of octaves), mean N and mean padded K per problem),
// for batches of at least 4 GFLOP, is timed once per
// process with every tile width (CUDA events; one warm-up run, best of two); a width replaces the
// cost model's choice when it is at least 10 % faster, and the choice is cached and used for every
// later batch of that class.  Only batches that may run repeatedly are timed (no accumulation
// into C, C distinct from A and B); the others use the cost model above.
struct TuneKey {
    int t, c, lf, ln, lk;
    bool operator<(const TuneKey& o) const {
        return std::tie(t, c, lf, ln, lk) < std::tie(o.t, o.c, o.lf, o.ln, o.lk);
    }
};
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tune;
std::atomic<long long> g_tune_changed{0};

TuneKey tune_key(const GemmBatch& g, Num t, Num cnum) {
    double n = 0.0, k = 0.0;
    for (const auto& p : g.probs) {
        n += p.N;
        for (int s = 0; s < p.nseg; ++s) k += (double)((g.segs[p.seg0 + s].K + 63) / 64) * 64;
    }
    const double np = (double)g.probs.size();
    auto lg = [](double x) { return (int)std::lround(std::log2(std::max(1.0, x))); };
    return {(int)t, (int)cnum, lg(g.flops) / 2, lg(n / np), lg(k / np)};
}

}  // namespace

void tune_stats(long long* classes, long long* changed) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    *classes = (long long)g_tune.size();
    *changed = g_tune_changed.load();
}

bool tc_available() {
    int dev = 0, major = 0, minor = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess) return false;
    if (cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess) return false;
    return major == 10 && minor == 3 && encode_fn() != nullptr;
}

namespace {
// One launch of the batch with tile width bn (its tile list uploaded for that width).
void launch_bn(GemmBatch& g, int bn, Num t, const void* A, long long a_rows, int lda, const void* B, long long b_rows,
               int ldb, void* C, Num cnum, unsigned* err, cudaStream_t st) {
    g.upload_tiles(BM, bn, st);
    const CUtensorMap ma = make_map(t, A, a_rows, lda, BM);
    const CUtensorMap mb = make_map(t, B, b_rows, ldb, bn);
    const bool bf = t == Num::BF16;
#define PD_TC(KIND, BN, ST)                                                                       \
    do {                                                                                          \
        if (cnum == Num::F64) launch_tc<KIND, BN, ST, double>(g, ma, mb, lda, ldb, C, err, st);   \
        else if (cnum == Num::F32) launch_tc<KIND, BN, ST, float>(g, ma, mb, lda, ldb, C, err, st); \
        else launch_tc<KIND, BN, ST, __nv_bfloat16>(g, ma, mb, lda, ldb, C, err, st);             \
    } while (0)
    if (bn == 256) {
        if (bf) PD_TC(0, 256, 4); else PD_TC(1, 256, 4);
    } else if (bn == 128) {
        if (bf) PD_TC(0, 128, 6); else PD_TC(1, 128, 6);
    } else {
        if (bf) PD_TC(0, 64, 8); else PD_TC(1, 64, 8);
    }
#undef PD_TC
}
}  // namespace

void run_gemm_tc(GemmBatch& g, Num t, const void* A, long long a_rows, int lda, const void* B, long long b_rows,
                 int ldb, void* C, Num cnum, unsigned* err, cudaStream_t st) {
    if (g.empty()) return;
    PD_REQUIRE(t == Num::BF16 || t == Num::F32, DMRG_ERR_ARG, "tensor-core operands must be bf16 or fp32");
    PD_REQUIRE(err != nullptr, DMRG_ERR_ARG, "tensor-core GEMM needs a device error word");
    for (const auto& p : g.probs)
        PD_REQUIRE(p.sak == 1 && p.sbk == 1 && p.sam == lda && p.sbn == ldb && p.scm == 1, DMRG_ERR_ARG,
                   "tensor-core GEMM needs K-major slabs with uniform leading dimensions");
    int bn = g.bn_choice;
    if (!bn) {
        const int model = pick_bn(g, (int)num_size(t));
        // small batches: timing noise exceeds any difference between widths
        bool repeatable = C != A && C != B && g.flops >= 4e9;
        for (const auto& p : g.probs) repeatable = repeatable && !p.accumulate;
        const TuneKey key = tune_key(g, t, cnum);
        int cached = 0;
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_tune.find(key);
            if (it != g_tune.end()) cached = it->second;
        }
        if (cached) {
            bn = cached;
        } else if (repeatable) {
            float best = -1.f;
            int best_bn = model;
            const int saved = g_prof_class;
            g_prof_class = PROF_NONE;   // trial runs are not tallied
            cudaEvent_t e0, e1;
            PD_CK(cudaEventCreate(&e0));
            PD_CK(cudaEventCreate(&e1));
            float model_ms = -1.f;
            for (int cand : {256, 128, 64}) {
                // one untimed run (tile list, descriptors, caches), then the best of two timed runs
                launch_bn(g, cand, t, A, a_rows, lda, B, b_rows, ldb, C, cnum, err, st);
                float ms = -1.f;
                for (int rep = 0; rep < 2; ++rep) {
                    PD_CK(cudaEventRecord(e0, st));
                    launch_bn(g, cand, t, A, a_rows, lda, B, b_rows, ldb, C, cnum, err, st);
                    PD_CK(cudaEventRecord(e1, st));
                    PD_CK(cudaEventSynchronize(e1));
                    float m = 0.f;
                    PD_CK(cudaEventElapsedTime(&m, e0, e1));
                    if (ms < 0.f || m < ms) ms = m;
                }
                if (cand == model) model_ms = ms;
                if (best < 0.f || ms < best) { best = ms; best_bn = cand; }
            }
            // keep the cost model's width unless a measured one is clearly faster (timing noise)
            if (model_ms >= 0.f && best > 0.9f * model_ms) best_bn = model;
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            g_prof_class = saved;
            {
                std::lock_guard<std::mutex> lk(g_tune_mu);
                g_tune[key] = best_bn;
            }
            if (best_bn != model) g_tune_changed.fetch_add(1);
            bn = best_bn;
        } else {
            bn = model;
        }
        g.bn_choice = bn;
    }
    launch_bn(g, bn, t, A, a_rows, lda, B, b_rows, ldb, C, cnum, err, st);
}

}  // namespace pd
