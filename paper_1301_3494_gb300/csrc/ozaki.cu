// FP64-accurate grouped GEMM on the bf16 tensor cores (error-free splitting in the manner of
// Ozaki, Ogita and Oishi, "Error-free transformations of matrix multiplication by using fast
// routines of matrix multiplication and its applications", Numer. Algorithms 59 (2012)).
//
// Same contract as the FP64 SIMT GEMM (internal.h):
//   C(m, n) (+)= alpha * sum_seg sum_k A(m, k) B(n, k).
// Every operand row is scaled by a power of two 2^e (|entries| < 2^e) and cut into s slices of
// beta bits each, x = 2^e sum_i a_i 2^(-i beta) + r with integer a_i, |a_i| < 2^beta (exact in
// bf16 for beta <= 8) and |r| < 2^(e - s beta).  A product of slices summed over k is a sum of
// integers below 2^24 when (2^beta - 1)^2 * (terms per accumulator) <= 2^24, so the tensor cores'
// FP32 accumulation of it is exact.  The slice pairs (i, j) with i + j <= s + 1 are formed on the
// tensor cores (one launch of the existing tcgen05 GEMM over all problems and pairs, FP32
// output) and combined in FP64 with their scales 2^(eA + eB - (i + j) beta).  The dropped pairs
// and the slice remainders contribute below (s^2/2 + 2) 2^(-s beta) max|A(m,:)| max|B(n,:)| per
// term; s = ceil(56 / beta) puts that at the level of FP64 rounding.
//
// Rows that meet in one accumulator must share their scale: the rows of all segments of one
// problem that produce the same output row (and column) are merged into one scale class
// (union-find over operand rows), and a class's exponent is that of its largest entry.  Operand
// blocks are stored once however many problems use them, so a class can also hold rows of other
// problems; the error bound then refers to the class maximum instead of the problem's own.  Before
// any slicing, a check compares, for every problem and output row (column), the exponent of its
// own largest operand entry with its class exponent; a gap above kGuardBits, or a NaN/Inf operand,
// sends the whole batch to the FP64 units (which also propagate NaN and Inf as FP64 would).
//
// Accumulators: one per slice pair ("pair" mode) or one per pair level i + j ("level" mode,
// fewer FP32 outputs, but more terms per accumulator and so a smaller beta); the mode and beta
// come from a cost model of the batch.  Batches whose K is too large for beta >= 2 use the FP64
// SIMT GEMM.
#include <cmath>
#include <numeric>
#include <unordered_map>

#include "plans.h"

namespace pd {

thread_local int g_gemm64_emu = 0;

struct EmuPlan {
    size_t nprobs = 0;                 // batch size the plan was built for
    unsigned long long key = 0;        // hash of the batch's problems and segments
    bool usable = false;
    int beta = 0, s = 0, ngroups = 0;
    int lda = 64, ldb = 64;
    long long a_rows = 0, b_rows = 0;  // slab rows per slice plane
    long long tmp_elems = 0;
    int nsplit_chunks = 0, ncomb_chunks = 0, na_cls = 0, nb_cls = 0;
    GemmBatch tc;
    DBuf split, comb, chunks_s, chunks_c, cls_a, cls_b, cmax, slab_a, slab_b, tmp, gshift, err;
    DBuf rowmax, chk, chk_rows, flag;  // per-row maxima, per-problem check jobs, guard flag
    int nchk = 0;
    double hi_unit = 1.0, lo_unit = 1.0;   // 2^(-l_mid beta), 2^(-(s+1) beta)
    double est_ms = 0.0;
};

}  // namespace pd

using namespace pd;

namespace {

// one operand block to slice: rows m < M of A[src + m*sm + k*sk], k < K; slab rows row0 + m
struct SplitJob {
    long long src, row0;
    int sm, sk, M, K;
    int which, pad_;         // 0: A operand, 1: B operand
};
// a chunk of up to kChunk elements of a job's M x ld region
struct Chunk {
    int job, e0, len, pad_;
};
// recombination of one original problem
struct CombJob {
    long long c_off, tmp_off, rowA0, rowB0;
    int M, N, scm, scn;
    int accumulate, pad_;
    double alpha;
};
constexpr int kChunk = 16384;
// largest gap (bits) between a problem's own row maximum and its scale class maximum
constexpr int kGuardBits = 3;

__device__ __forceinline__ unsigned long long abs_bits(double x) {
    return (unsigned long long)__double_as_longlong(fabs(x));
}

// exponent e of a class maximum mx = f 2^e, f in [0.5, 1) (every entry of the class is below 2^e)
__device__ __forceinline__ int class_exp(unsigned long long bits) {
    const int E = (int)((bits >> 52) & 0x7FF);
    if (E != 0) return E - 1022;
    int e = 0;
    const double mx = __longlong_as_double((long long)bits);
    if (mx > 0.0) frexp(mx, &e);          // subnormal maximum
    return e;
}

// row maxima: rowmax[side_base + row] = max |x| over the row's K entries (bit patterns of
// nonnegative doubles order like unsigned integers; A rows first, then B rows).  Chunks start at
// multiples of kChunk and rows are ld (a multiple of 64) long, so the 32 elements a warp takes at a
// time lie in one row: one atomic per warp.
__global__ void k_oz_absmax(const SplitJob* __restrict__ jobs, const Chunk* __restrict__ chunks,
                            const double* __restrict__ A, const double* __restrict__ B, long long a_rows,
                            unsigned long long* __restrict__ rowmax, int ld_a, int ld_b) {
    const Chunk c = chunks[blockIdx.x];
    const SplitJob j = jobs[c.job];
    const double* X = j.which ? B : A;
    unsigned long long* mx = rowmax + (j.which ? a_rows : 0);
    const int ld = j.which ? ld_b : ld_a;
    const int lane = threadIdx.x & 31;
    for (int base = threadIdx.x - lane; base < c.len; base += blockDim.x) {      // c.len: a multiple of 64
        const int idx = c.e0 + base + lane;
        const int m = idx / ld, k = idx % ld;
        unsigned long long v = 0;
        if (k < j.K) v = abs_bits(X[j.src + (long long)m * j.sm + (long long)k * j.sk]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
            v = w > v ? w : v;
        }
        if (lane == 0 && v != 0) atomicMax(mx + j.row0 + m, v);
    }
}

// class maxima from row maxima (cmax[cls[r]] over the rows of both sides; B classes follow the
// na_cls A classes); a NaN or Inf anywhere (exponent field 0x7FF) sets bit 2 of *flag.
__global__ void k_oz_classmax(const unsigned long long* __restrict__ rowmax, long long a_rows, long long rows,
                              const int* __restrict__ cls_a, const int* __restrict__ cls_b, int na_cls,
                              unsigned long long* __restrict__ cmax, unsigned* __restrict__ flag) {
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < rows; r += (long long)gridDim.x * blockDim.x) {
        const unsigned long long v = rowmax[r];
        if (v == 0) continue;
        if (((v >> 52) & 0x7FF) == 0x7FF) atomicOr(flag, 2u);
        const int c = r < a_rows ? cls_a[r] : na_cls + cls_b[r - a_rows];
        atomicMax(cmax + c, v);
    }
}

// one output row (A side) or column (B side) of one problem: the slab rows of its segments
struct ChkJob {
    int n, nseg, seg0, which;   // rows (M or N), segments, first entry in chk_rows, side
};
// For every row m of a job: own = max over its segments of rowmax[row0_s + m]; a class exponent
// more than guard bits above own's sets bit 1 of *flag (the batch then runs on the FP64 units).
__global__ void k_oz_check(const ChkJob* __restrict__ jobs, const long long* __restrict__ chk_rows,
                           const unsigned long long* __restrict__ rowmax, long long a_rows,
                           const int* __restrict__ cls_a, const int* __restrict__ cls_b, int na_cls,
                           const unsigned long long* __restrict__ cmax, int guard, unsigned* __restrict__ flag) {
    const ChkJob j = jobs[blockIdx.x];
    const long long base = j.which ? a_rows : 0;
    for (int m = threadIdx.x; m < j.n; m += blockDim.x) {
        unsigned long long own = 0;
        for (int s = 0; s < j.nseg; ++s) {
            const unsigned long long v = rowmax[base + chk_rows[j.seg0 + s] + m];
            own = v > own ? v : own;
        }
        if (own == 0) continue;          // an all-zero row contributes nothing
        const long long r0 = chk_rows[j.seg0] + m;
        const unsigned long long cm = cmax[j.which ? na_cls + cls_b[r0] : cls_a[r0]];
        if (class_exp(cm) - class_exp(own) > guard) atomicOr(flag, 1u);
    }
}

// slices: slab[(i * rows + row0 + m) * ld + k] = a_i for k < K, 0 for K <= k < ld.  Integer
// arithmetic on the FP64 bit pattern (the FP64 units are slow on this part): with x = +-mant
// 2^(E - 1075) and the class exponent e, |x| 2^(62 - e) = R is a 62-bit fixed-point integer and
// the slices are its consecutive beta-bit fields from the top, a_i = sign(x) field_i -- the
// digits of the truncated expansion x 2^-e = sum_i a_i 2^(-i beta) + r.
__global__ void k_oz_split(const SplitJob* __restrict__ jobs, const Chunk* __restrict__ chunks,
                           const double* __restrict__ A, const double* __restrict__ B, const int* __restrict__ cls_a,
                           const int* __restrict__ cls_b, int na_cls, const unsigned long long* __restrict__ cmax,
                           __nv_bfloat16* __restrict__ slab_a, __nv_bfloat16* __restrict__ slab_b, long long rows_a,
                           long long rows_b, int ld_a, int ld_b, int s, int beta) {
    const Chunk c = chunks[blockIdx.x];
    const SplitJob j = jobs[c.job];
    const double* X = j.which ? B : A;
    const int* cls = j.which ? cls_b : cls_a;
    const unsigned long long* mx = cmax + (j.which ? na_cls : 0);
    __nv_bfloat16* slab = j.which ? slab_b : slab_a;
    const long long plane = (j.which ? rows_b : rows_a) * (long long)(j.which ? ld_b : ld_a);
    const int ld = j.which ? ld_b : ld_a;
    const unsigned long long fmask = (1ull << beta) - 1ull;
    for (int e = threadIdx.x; e < c.len; e += blockDim.x) {
        const int idx = c.e0 + e;
        const int m = idx / ld, k = idx % ld;
        __nv_bfloat16* out = slab + (j.row0 + m) * ld + k;
        unsigned long long R = 0;
        bool neg = false;
        if (k < j.K) {
            const unsigned long long bits = (unsigned long long)__double_as_longlong(
                X[j.src + (long long)m * j.sm + (long long)k * j.sk]);
            neg = (bits >> 63) != 0;
            const int E = (int)((bits >> 52) & 0x7FF);
            unsigned long long mant = bits & ((1ull << 52) - 1ull);
            int Eu = E;
            if (E != 0) mant |= (1ull << 52);
            else Eu = 1;                                   // zero or subnormal
            const int sh = Eu - class_exp(mx[cls[j.row0 + m]]) - 1013;   // R = mant 2^sh, sh <= 9
            if (mant != 0) R = sh >= 0 ? (mant << sh) : (sh > -64 ? (mant >> (-sh)) : 0ull);
        }
        for (int i = 1; i <= s; ++i) {
            const int f = (int)((R >> (62 - i * beta)) & fmask);
            out[(i - 1) * plane] = __int2bfloat16_rn(neg ? -f : f);      // |f| < 256: exact
        }
    }
}

// C(m, n) (+)= alpha 2^(eA + eB) sum_g tmp_g(m, n) 2^(-l_g beta).  Every tmp_g is an integer below
// 2^24 (exact in FP32); the sum is formed exactly in two 64-bit fixed-point accumulators -- levels
// l <= l_mid in units of 2^(-l_mid beta), the rest in units of 2^(-(s+1) beta) -- and converted
// to FP64 once (integer arithmetic: the FP64 units are slow on this part).  gshift[g] >= 0 is
// the left shift of group g into its accumulator, negative (-1 - shift) for the low one.
__global__ void k_oz_combine(const CombJob* __restrict__ jobs, const Chunk* __restrict__ chunks,
                             const float* __restrict__ tmp, const int* __restrict__ gshift, int ngroups,
                             double hi_unit, double lo_unit, const int* __restrict__ cls_a,
                             const int* __restrict__ cls_b, int na_cls, const unsigned long long* __restrict__ cmax,
                             double* __restrict__ C) {
    const Chunk c = chunks[blockIdx.x];
    const CombJob j = jobs[c.job];
    const long long mn = (long long)j.M * j.N;
    for (int e = threadIdx.x; e < c.len; e += blockDim.x) {
        const int idx = c.e0 + e;
        const int m = idx % j.M, n = idx / j.M;
        long long hi = 0, lo = 0;
        const float* t = tmp + j.tmp_off + idx;
        for (int g = 0; g < ngroups; ++g) {
            const long long v = (long long)__float2int_rz(t[g * mn]);
            const int sh = gshift[g];
            if (sh >= 0) hi += v << sh;
            else lo += v << (-1 - sh);
        }
        double v = (double)hi * hi_unit + (double)lo * lo_unit;
        const int ex = class_exp(cmax[cls_a[j.rowA0 + m]]) + class_exp(cmax[na_cls + cls_b[j.rowB0 + n]]);
        v = j.alpha * ldexp(v, ex);
        double* dst = C + j.c_off + (long long)m * j.scm + (long long)n * j.scn;
        *dst = j.accumulate ? *dst + v : v;
    }
}

struct UF {
    std::vector<int> p;
    explicit UF(size_t n) : p(n) { std::iota(p.begin(), p.end(), 0); }
    int find(int x) {
        while (p[x] != x) x = p[x] = p[p[x]];
        return x;
    }
    void join(int a, int b) {
        a = find(a);
        b = find(b);
        if (a != b) p[std::max(a, b)] = std::min(a, b);
    }
};

struct BlockKey {
    long long off;
    int sm, sk, K;
    bool operator==(const BlockKey& o) const { return off == o.off && sm == o.sm && sk == o.sk && K == o.K; }
};
struct BlockKeyHash {
    size_t operator()(const BlockKey& k) const {
        return std::hash<long long>()(k.off * 1000003LL + k.sm * 131LL + k.sk * 7LL + k.K);
    }
};

// Operand blocks of one side, deduplicated; slab rows assigned consecutively per block.
struct Side {
    std::unordered_map<BlockKey, int, BlockKeyHash> index;
    std::vector<BlockKey> keys;
    std::vector<int> rows;          // rows per block (max M seen)
    std::vector<long long> row0;
    int block(const BlockKey& k, int M) {
        auto it = index.find(k);
        if (it != index.end()) {
            rows[it->second] = std::max(rows[it->second], M);
            return it->second;
        }
        const int id = (int)keys.size();
        index.emplace(k, id);
        keys.push_back(k);
        rows.push_back(M);
        return id;
    }
    long long layout() {
        row0.assign(keys.size(), 0);
        long long r = 0;
        for (size_t i = 0; i < keys.size(); ++i) {
            row0[i] = r;
            r += rows[i];
        }
        return r;
    }
};

void chunk_jobs(const std::vector<long long>& sizes, std::vector<Chunk>& out) {
    for (size_t j = 0; j < sizes.size(); ++j)
        for (long long e = 0; e < sizes[j]; e += kChunk)
            out.push_back({(int)j, (int)e, (int)std::min<long long>(kChunk, sizes[j] - e), 0});
}

// FNV-1a over the problem and segment lists: a plan is reused only for the batch it was built for.
unsigned long long batch_key(const GemmBatch& g) {
    unsigned long long h = 1469598103934665603ull;
    auto mix = [&](const void* p, size_t n) {
        const unsigned char* b = static_cast<const unsigned char*>(p);
        for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
    };
    if (!g.probs.empty()) mix(g.probs.data(), g.probs.size() * sizeof(GProb));
    if (!g.segs.empty()) mix(g.segs.data(), g.segs.size() * sizeof(GSeg));
    return h;
}

std::unique_ptr<EmuPlan> build_plan(const GemmBatch& g, cudaStream_t st) {
    std::unique_ptr<EmuPlan> P(new EmuPlan());
    P->nprobs = g.probs.size();
    P->key = batch_key(g);
    Side sa, sb;
    std::vector<std::vector<int>> pa(g.probs.size()), pb(g.probs.size());   // block ids per segment
    long long kmax_tot = 0;
    int kmax = 1;
    double flops = 0.0, mn_tot = 0.0, tiles = 0.0;
    for (size_t p = 0; p < g.probs.size(); ++p) {
        const GProb& q = g.probs[p];
        long long kt = 0;
        for (int s = 0; s < q.nseg; ++s) {
            const GSeg& sg = g.segs[q.seg0 + s];
            pa[p].push_back(sa.block({sg.a_off, q.sam, q.sak, sg.K}, q.M));
            pb[p].push_back(sb.block({sg.b_off, q.sbn, q.sbk, sg.K}, q.N));
            kt += sg.K;
            kmax = std::max(kmax, sg.K);
            flops += 2.0 * q.M * q.N * sg.K;
        }
        kmax_tot = std::max(kmax_tot, kt);
        mn_tot += (double)q.M * q.N;
        tiles += (double)((q.M + 127) / 128) * ((q.N + 127) / 128);
    }
    P->a_rows = sa.layout();
    P->b_rows = sb.layout();
    PD_REQUIRE(P->a_rows < (long long)INT32_MAX && P->b_rows < (long long)INT32_MAX, DMRG_ERR_CAPACITY,
               "emulated GEMM batch too large");
    // scale classes: rows feeding one output row (column) of one problem share a class
    UF ua((size_t)std::max<long long>(1, P->a_rows)), ub((size_t)std::max<long long>(1, P->b_rows));
    for (size_t p = 0; p < g.probs.size(); ++p) {
        const GProb& q = g.probs[p];
        for (size_t s = 1; s < pa[p].size(); ++s) {
            if (pa[p][s] != pa[p][0])
                for (int m = 0; m < q.M; ++m) ua.join((int)(sa.row0[pa[p][0]] + m), (int)(sa.row0[pa[p][s]] + m));
            if (pb[p][s] != pb[p][0])
                for (int n = 0; n < q.N; ++n) ub.join((int)(sb.row0[pb[p][0]] + n), (int)(sb.row0[pb[p][s]] + n));
        }
    }
    auto classes = [](UF& u, long long n, int* ncls) {
        std::vector<int> c((size_t)std::max<long long>(1, n), 0), id((size_t)std::max<long long>(1, n), -1);
        int k = 0;
        for (long long r = 0; r < n; ++r) {
            const int root = u.find((int)r);
            if (id[root] < 0) id[root] = k++;
            c[r] = id[root];
        }
        *ncls = std::max(1, k);
        return c;
    };
    const std::vector<int> ca = classes(ua, P->a_rows, &P->na_cls), cb = classes(ub, P->b_rows, &P->nb_cls);
    // guard jobs: every problem's output rows (A side) and columns (B side)
    std::vector<ChkJob> chk;
    std::vector<long long> chk_rows;
    for (size_t p = 0; p < g.probs.size(); ++p) {
        const GProb& q = g.probs[p];
        chk.push_back({q.M, (int)pa[p].size(), (int)chk_rows.size(), 0});
        for (int b : pa[p]) chk_rows.push_back(sa.row0[b]);
        chk.push_back({q.N, (int)pb[p].size(), (int)chk_rows.size(), 1});
        for (int b : pb[p]) chk_rows.push_back(sb.row0[b]);
    }
    // mode and beta
    struct Opt { bool level; int beta, s, groups, pairs; double ms; };
    Opt best{false, 0, 0, 0, 0, -1.0};
    for (int lv = 0; lv < 2; ++lv)
        for (int beta = 8; beta >= 2; --beta) {
            const int s = (56 + beta - 1) / beta;
            const double per = lv ? (double)s : 1.0;
            const double lim = (double)(1 << 24);
            if ((double)((1 << beta) - 1) * ((1 << beta) - 1) * (double)kmax_tot * per > lim) continue;
            const int pairs = s * (s + 1) / 2, groups = lv ? s : pairs;
            // tensor-core flops, FP32 partial results written and read back, per-tile overhead
            const double ms = pairs * flops / 2.5e11 + groups * mn_tot * 8.0 / 5.0e9 + groups * tiles * 1.5e-3 / 152.0;
            if (best.ms < 0 || ms < best.ms) best = {lv != 0, beta, s, groups, pairs, ms};
            break;
        }
    if (best.ms < 0) return P;          // K too large for exact FP32 accumulation
    P->beta = best.beta;
    P->s = best.s;
    P->ngroups = best.groups;
    P->est_ms = best.ms;
    P->lda = (kmax + 63) / 64 * 64;
    P->ldb = P->lda;
    // groups: slice pairs (i, j), 1-based, i + j <= s + 1, and their shifts into the combine's
    // two fixed-point accumulators (levels <= l_mid in units of 2^(-l_mid beta), the rest in
    // units of 2^(-(s+1) beta)); both stay below 2^63 for every beta (see k_oz_combine)
    const int l_mid = std::min(P->s + 1, 2 + 36 / P->beta);
    P->hi_unit = std::ldexp(1.0, -l_mid * P->beta);
    P->lo_unit = std::ldexp(1.0, -(P->s + 1) * P->beta);
    std::vector<std::vector<std::pair<int, int>>> grp;
    std::vector<int> gshift;
    auto shift_of = [&](int l) { return l <= l_mid ? (l_mid - l) * P->beta : -1 - (P->s + 1 - l) * P->beta; };
    if (best.level) {
        for (int l = 2; l <= P->s + 1; ++l) {
            grp.emplace_back();
            for (int i = 1; i < l; ++i) grp.back().push_back({i, l - i});
            gshift.push_back(shift_of(l));
        }
    } else {
        for (int l = 2; l <= P->s + 1; ++l)
            for (int i = 1; i < l; ++i) {
                grp.push_back({{i, l - i}});
                gshift.push_back(shift_of(l));
            }
    }
    // tensor-core batch (FP32 out), combine jobs
    std::vector<CombJob> comb;
    std::vector<long long> csizes;
    std::vector<GSeg> segs;
    long long toff = 0;
    for (size_t p = 0; p < g.probs.size(); ++p) {
        const GProb& q = g.probs[p];
        const long long mn = (long long)q.M * q.N;
        for (int gi = 0; gi < P->ngroups; ++gi) {
            segs.clear();
            for (const auto& ij : grp[gi])
                for (int s = 0; s < q.nseg; ++s) {
                    const GSeg& sg = g.segs[q.seg0 + s];
                    segs.push_back({((long long)(ij.first - 1) * P->a_rows + sa.row0[pa[p][s]]) * P->lda,
                                    ((long long)(ij.second - 1) * P->b_rows + sb.row0[pb[p][s]]) * P->ldb, sg.K, 0});
                }
            P->tc.add(q.M, q.N, toff + gi * mn, P->lda, 1, P->ldb, 1, 1, q.M, segs);
        }
        comb.push_back({q.c_off, toff, sa.row0[pa[p][0]], sb.row0[pb[p][0]], q.M, q.N, q.scm, q.scn, q.accumulate, 0,
                        q.alpha});
        csizes.push_back(mn);
        toff += (long long)P->ngroups * mn;
    }
    P->tmp_elems = toff;
    // split jobs over both sides
    std::vector<SplitJob> jobs;
    std::vector<long long> ssizes;
    for (size_t b = 0; b < sa.keys.size(); ++b) {
        jobs.push_back({sa.keys[b].off, sa.row0[b], sa.keys[b].sm, sa.keys[b].sk, sa.rows[b], sa.keys[b].K, 0, 0});
        ssizes.push_back((long long)sa.rows[b] * P->lda);
    }
    for (size_t b = 0; b < sb.keys.size(); ++b) {
        jobs.push_back({sb.keys[b].off, sb.row0[b], sb.keys[b].sm, sb.keys[b].sk, sb.rows[b], sb.keys[b].K, 1, 0});
        ssizes.push_back((long long)sb.rows[b] * P->ldb);
    }
    std::vector<Chunk> sch, cch;
    chunk_jobs(ssizes, sch);
    chunk_jobs(csizes, cch);
    PD_REQUIRE(sch.size() < (size_t)INT32_MAX && cch.size() < (size_t)INT32_MAX &&
                   P->a_rows * P->s < (long long)INT32_MAX && P->b_rows * P->s < (long long)INT32_MAX,
               DMRG_ERR_CAPACITY, "emulated GEMM batch too large");
    P->nsplit_chunks = (int)sch.size();
    P->ncomb_chunks = (int)cch.size();
    upload(P->split, jobs, st);
    upload(P->comb, comb, st);
    upload(P->chunks_s, sch, st);
    upload(P->chunks_c, cch, st);
    upload(P->cls_a, ca, st);
    upload(P->cls_b, cb, st);
    upload(P->gshift, gshift, st);
    upload(P->chk, chk, st);
    upload(P->chk_rows, chk_rows, st);
    P->nchk = (int)chk.size();
    P->rowmax.ensure((size_t)std::max<long long>(1, P->a_rows + P->b_rows) * 8, st);
    P->flag.ensure(4, st);
    P->cmax.ensure((size_t)(P->na_cls + P->nb_cls) * 8, st);
    P->slab_a.ensure((size_t)std::max<long long>(1, P->a_rows * P->s) * P->lda * 2, st);
    P->slab_b.ensure((size_t)std::max<long long>(1, P->b_rows * P->s) * P->ldb * 2, st);
    P->tmp.ensure((size_t)std::max<long long>(1, P->tmp_elems) * 4, st);
    P->err.ensure(4, st);
    PD_CK(cudaMemsetAsync(P->err.p, 0, 4, st));
    P->usable = true;
    return P;
}

}  // namespace

namespace pd {

void check_err_word(unsigned* err, cudaStream_t st);

void free_emu_plan(EmuPlan* p) { delete p; }

bool run_gemm64_emu(GemmBatch& g, const double* A, const double* B, double* C, cudaStream_t st) {
    if (g.empty()) return true;
    if (!tc_available()) return false;
    const unsigned long long key = batch_key(g);
    if (!g.emu || g.emu->nprobs != g.probs.size() || g.emu->key != key)
        g.emu.reset(build_plan(g, st).release(), free_emu_plan);
    EmuPlan& P = *g.emu;
    if (!P.usable) return false;
    const int cls = g_prof_class == PROF_ENV ? PROF_ENV : PROF_F64;
    void* tok = prof_on() ? prof_start(st) : nullptr;
    PD_CK(cudaMemsetAsync(P.rowmax.p, 0, (size_t)std::max<long long>(1, P.a_rows + P.b_rows) * 8, st));
    PD_CK(cudaMemsetAsync(P.cmax.p, 0, (size_t)(P.na_cls + P.nb_cls) * 8, st));
    PD_CK(cudaMemsetAsync(P.flag.p, 0, 4, st));
    PD_CK(cudaMemsetAsync(P.err.p, 0, 4, st));
    k_oz_absmax<<<(unsigned)P.nsplit_chunks, 256, 0, st>>>(P.split.as<SplitJob>(), P.chunks_s.as<Chunk>(), A, B,
                                                           P.a_rows, P.rowmax.as<unsigned long long>(), P.lda, P.ldb);
    PD_LAUNCHED();
    const long long rows = P.a_rows + P.b_rows;
    k_oz_classmax<<<(unsigned)std::min<long long>(1024, (rows + 255) / 256), 256, 0, st>>>(
        P.rowmax.as<unsigned long long>(), P.a_rows, rows, P.cls_a.as<int>(), P.cls_b.as<int>(), P.na_cls,
        P.cmax.as<unsigned long long>(), P.flag.as<unsigned>());
    PD_LAUNCHED();
    k_oz_check<<<(unsigned)P.nchk, 128, 0, st>>>(P.chk.as<ChkJob>(), P.chk_rows.as<long long>(),
                                                 P.rowmax.as<unsigned long long>(), P.a_rows, P.cls_a.as<int>(),
                                                 P.cls_b.as<int>(), P.na_cls, P.cmax.as<unsigned long long>(),
                                                 kGuardBits, P.flag.as<unsigned>());
    PD_LAUNCHED();
    unsigned flag = 0;
    PD_CK(cudaMemcpyAsync(&flag, P.flag.p, 4, cudaMemcpyDeviceToHost, st));
    PD_CK(cudaStreamSynchronize(st));
    if (flag) {
        // a class maximum far above a problem's own, or a non-finite operand: FP64 units
        if (tok) prof_stop(tok, st, PROF_NONE, 0.0);
        prof_emu_fallback();
        return false;
    }
    k_oz_split<<<(unsigned)P.nsplit_chunks, 256, 0, st>>>(
        P.split.as<SplitJob>(), P.chunks_s.as<Chunk>(), A, B, P.cls_a.as<int>(), P.cls_b.as<int>(), P.na_cls,
        P.cmax.as<unsigned long long>(), P.slab_a.as<__nv_bfloat16>(), P.slab_b.as<__nv_bfloat16>(), P.a_rows,
        P.b_rows, P.lda, P.ldb, P.s, P.beta);
    PD_LAUNCHED();
    const int saved = g_prof_class;
    g_prof_class = PROF_NONE;      // tallied once below, as the FP64 GEMM it stands for
    run_gemm_tc(P.tc, Num::BF16, P.slab_a.p, P.a_rows * P.s, P.lda, P.slab_b.p, P.b_rows * P.s, P.ldb, P.tmp.p,
                Num::F32, P.err.as<unsigned>(), st);
    g_prof_class = saved;
    k_oz_combine<<<(unsigned)P.ncomb_chunks, 256, 0, st>>>(P.comb.as<CombJob>(), P.chunks_c.as<Chunk>(),
                                                           P.tmp.as<float>(), P.gshift.as<int>(), P.ngroups,
                                                           P.hi_unit, P.lo_unit,
                                                           P.cls_a.as<int>(), P.cls_b.as<int>(), P.na_cls,
                                                           P.cmax.as<unsigned long long>(), C);
    PD_LAUNCHED();
    if (tok) prof_stop(tok, st, cls, g.flops);
    check_err_word(P.err.as<unsigned>(), st);
    return true;
}

void emu_plan_info(const GemmBatch& g, int* beta, int* s, int* groups) {
    if (!g.emu || !g.emu->usable) { *beta = *s = *groups = 0; return; }
    *beta = g.emu->beta;
    *s = g.emu->s;
    *groups = g.emu->ngroups;
}

}  // namespace pd
