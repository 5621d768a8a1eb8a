// Block layouts, contraction plans and the device-side building blocks of one two-site step.
#pragma once
#include <algorithm>
#include <memory>
#include <vector>

#include "internal.h"

namespace pd {

// ------------------------------------------------------------------------------------------
// U(1) sectors of one bond (ascending charges)
// ------------------------------------------------------------------------------------------
struct Sec {
    std::vector<int> q, m;
    int n() const { return (int)q.size(); }
    int find(int x) const {
        auto it = std::lower_bound(q.begin(), q.end(), x);
        if (it == q.end() || *it != x) return -1;
        return (int)(it - q.begin());
    }
    int maxm() const {
        int r = 0;
        for (int v : m) r = std::max(r, v);
        return r;
    }
    long long total() const {
        long long t = 0;
        for (int v : m) t += v;
        return t;
    }
    bool operator==(const Sec& o) const { return q == o.q && m == o.m; }
};

// MPO of one site on the host: W[w][s][s'][w'] and the fluxes of both bonds.
struct SiteMPO {
    int Dl = 0, Dr = 0, d = 0;
    std::vector<double> W;
    std::vector<int> fl, fr;
    double at(int w, int s, int sp, int wp) const {
        return W[(((size_t)w * d + s) * d + sp) * Dr + wp];
    }
};

// ------------------------------------------------------------------------------------------
// Device buffers (stream-ordered allocator)
// ------------------------------------------------------------------------------------------
struct DBuf {
    void* p = nullptr;
    size_t bytes = 0;
    cudaStream_t st = nullptr;
    DBuf() = default;
    DBuf(const DBuf&) = delete;
    DBuf& operator=(const DBuf&) = delete;
    DBuf(DBuf&& o) noexcept { *this = std::move(o); }
    DBuf& operator=(DBuf&& o) noexcept {
        if (this != &o) {
            release();
            p = o.p; bytes = o.bytes; st = o.st;
            o.p = nullptr; o.bytes = 0;
        }
        return *this;
    }
    ~DBuf() { release(); }
    void release() {
        if (p) cudaFreeAsync(p, st);
        p = nullptr;
        bytes = 0;
    }
    // (Re)allocate at least `b` bytes on stream s; contents undefined after growth.
    void ensure(size_t b, cudaStream_t s) {
        if (b == 0) b = 16;
        if (p && bytes >= b) { st = s; return; }
        release();
        PD_CK(cudaMallocAsync(&p, b, s));
        bytes = b;
        st = s;
    }
    template <class T> T* as() const { return reinterpret_cast<T*>(p); }
    // Hand the buffer to another stream: later frees are ordered after that stream's work.
    void rebind(cudaStream_t s) { st = s; }
};

template <class T>
inline void upload(DBuf& d, const std::vector<T>& h, cudaStream_t st) {
    d.ensure(h.size() * sizeof(T), st);
    if (!h.empty()) PD_CK(cudaMemcpyAsync(d.p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, st));
}

// ------------------------------------------------------------------------------------------
// Block layouts
// ------------------------------------------------------------------------------------------
struct SiteLayout {            // packed site tensor: blocks (i, s) -> [m_i][m_j]
    struct B { int i, s, j; long long off; int rows, cols; };
    std::vector<B> blk;
    std::vector<int> index;    // i*d + s -> block or -1
    long long size = 0;
    int d = 0;
    int at(int i, int s) const { return index[(size_t)i * d + s]; }
};
SiteLayout site_layout(const Sec& bl, const Sec& br, const std::vector<int>& qn);

struct PsiLayout {             // packed two-site: blocks (i, s1, s2) -> [m_i][m_k]
    struct B { int i, s1, s2, k; long long off; int rows, cols; };
    std::vector<B> blk;
    std::vector<int> index;    // (i*d1 + s1)*d2 + s2 -> block or -1
    long long size = 0;
    int d = 0, d1 = 0, d2 = 0;
    int at(int i, int s1, int s2) const { return index[((size_t)i * d1 + s1) * d2 + s2]; }
};
PsiLayout psi_layout(const Sec& bl, const Sec& br, const std::vector<int>& qn);
// Two legs with different local charge lists (d1 = qn1.size(), d2 = qn2.size()).
PsiLayout psi_layout2(const Sec& bl, const Sec& br, const std::vector<int>& qn1, const std::vector<int>& qn2);

struct EnvLayout {             // environment slab: blocks (bra i, w) -> rows [row, row+m_i), ket k
    struct B { int i, w, k; long long row; long long packed; int rows, cols; };
    std::vector<B> blk;
    std::vector<int> index;    // i*D + w -> block or -1
    int D = 0, ld = 0;
    long long rows = 0, packed_size = 0;
    int at(int i, int w) const { return index[(size_t)i * D + w]; }
};
EnvLayout env_layout(const Sec& b, const std::vector<int>& flux, int ld);

// Element type used for the tensor-core operand slabs and the row padding they need.
enum class Num { F64, F32, BF16 };
inline size_t num_size(Num t) { return t == Num::F64 ? 8 : (t == Num::F32 ? 4 : 2); }
// Internal matvec arithmetic for the accurate Davidson refinement of the mixed modes: FP32
// operands and accumulation on the CUDA cores (same slab layout as TF32).
constexpr int PREC_F32 = 3;
// Environment arithmetic of the mixed modes with FP64-accurate environments: the tensor-core
// operand layout (rows and leading dimension padded to 64), FP64 storage, FP64 GEMMs.
constexpr int PREC_ENV64 = 4;
inline int pad_ld(int x, int prec) {
    int a = (prec == DMRG_FP64) ? 2 : 64;
    x = std::max(x, 1);
    return (x + a - 1) / a * a;
}
inline int kpad(int K, int prec) { return prec == DMRG_FP64 ? K : (K + 63) / 64 * 64; }
// Operand types per precision: matvec operands / environment-update operands / env storage.
inline Num mv_num(int prec) {
    return prec == DMRG_FP64 ? Num::F64 : ((prec == DMRG_TF32 || prec == PREC_F32) ? Num::F32 : Num::BF16);
}
inline Num env_num(int prec) { return (prec == DMRG_FP64 || prec == PREC_ENV64) ? Num::F64 : Num::F32; }

// ------------------------------------------------------------------------------------------
// Grouped GEMM batch (host list -> device arrays -> FP64 SIMT or tcgen05 launch)
// ------------------------------------------------------------------------------------------
struct EmuPlan;
// FP64 GEMMs through the bf16 tensor cores (ozaki.cu) when set on the calling thread.
extern thread_local int g_gemm64_emu;
struct GemmBatch {
    std::vector<GProb> probs;
    std::vector<GSeg> segs;
    double flops = 0.0;
    // device copies
    DBuf dprobs, dsegs, dtiles;
    int ntiles = 0;
    int tile_m = 0, tile_n = 0;         // shape of the uploaded tile list
    int bn_choice = 0;                  // tensor-core tile width chosen for this batch (0: not yet)
    long long a_rows = 0, b_rows = 0;   // slab extents (tensor-core path)
    int lda = 0, ldb = 0;
    std::shared_ptr<EmuPlan> emu;       // plan of the FP64-emulated execution, built on first use

    void add(int M, int N, long long c_off, int sam, int sak, int sbn, int sbk, int scm, int scn,
             const std::vector<GSeg>& sg, int accumulate = 0, double alpha = 1.0) {
        if (M <= 0 || N <= 0 || sg.empty()) return;
        GProb p{};
        p.M = M; p.N = N; p.seg0 = (int)segs.size(); p.nseg = (int)sg.size();
        p.c_off = c_off; p.sam = sam; p.sak = sak; p.sbn = sbn; p.sbk = sbk; p.scm = scm; p.scn = scn;
        p.accumulate = accumulate; p.alpha = alpha;
        for (const auto& s : sg) {
            segs.push_back(s);
            flops += 2.0 * M * N * s.K;
        }
        probs.push_back(p);
    }
    bool empty() const { return probs.empty(); }
    // Upload for the FP64 engine (64x64 tiles) or the tensor-core engine (tile_m x tile_n).
    void upload_tiles(int tm, int tn, cudaStream_t st);
};

// Run a batch: FP64 SIMT (A, B, C double) or tensor core (A, B slabs of type `t`, C of type
// float or double per `c_is_f64`).
void run_gemm64(GemmBatch& g, const double* A, const double* B, double* C, cudaStream_t st);
void run_gemm32(GemmBatch& g, const float* A, const float* B, float* C, cudaStream_t st);
void run_gemm_tc(GemmBatch& g, Num t, const void* A, long long a_rows, int lda, const void* B,
                 long long b_rows, int ldb, void* C, Num cnum, unsigned* err, cudaStream_t st);
bool tc_available();
// Tile-width autotuner of the tensor-core GEMM: shape classes timed so far, and how many of them
// chose a different width than the cost model.
void tune_stats(long long* classes, long long* changed);
// FP64-accurate execution of an FP64 batch on the bf16 tensor cores (error-free slicing, exact
// FP32 accumulation, FP64 recombination).  Returns false, doing nothing, when the tensor cores
// are unavailable or the batch's K is too large for exact accumulation.  Synchronises (checks
// the tensor-core kernel's error word).
bool run_gemm64_emu(GemmBatch& g, const double* A, const double* B, double* C, cudaStream_t st);
void emu_plan_info(const GemmBatch& g, int* beta, int* s, int* groups);

// ------------------------------------------------------------------------------------------
// Generic job lists uploaded once, launched many times
// ------------------------------------------------------------------------------------------
struct CopyList {
    std::vector<CopyJob> jobs;
    std::vector<long long> elems;
    DBuf d, dc;
    int nchunks = 0;
    int max_elems = 0;
    void add(const CopyJob& j) {
        jobs.push_back(j);
        elems.push_back((long long)j.rows * std::max(j.cols, j.zero_to));
        max_elems = std::max(max_elems, j.rows * std::max(j.cols, j.zero_to));
    }
    void up(cudaStream_t st) {
        upload(d, jobs, st);
        std::vector<int2> c = make_chunks(elems);
        nchunks = (int)c.size();
        upload(dc, c, st);
    }
};
struct MixList {
    std::vector<MixJob> jobs;
    std::vector<MixTerm> terms;
    DBuf dj, dt, dc;
    int nchunks = 0;
    int max_elems = 0;
    double flops = 0.0;
    void up(cudaStream_t st) {
        upload(dj, jobs, st);
        upload(dt, terms, st);
        std::vector<long long> el;
        for (const auto& j : jobs) el.push_back((long long)j.rows * std::max(j.cols, j.zero_to));
        std::vector<int2> c = make_chunks(el);
        nchunks = (int)c.size();
        upload(dc, c, st);
    }
};

template <class Tin>
void run_copy(const CopyList& c, const Tin* src, void* dst, Num out, cudaStream_t st);
template <class Tin>
void run_mix(const MixList& m, const Tin* in, void* out, Num t, cudaStream_t st);

// ------------------------------------------------------------------------------------------
// Environment slab on the device
// ------------------------------------------------------------------------------------------
struct EnvSlab {
    EnvLayout lay;
    Num num = Num::F64;       // storage type (FP64 or FP32)
    DBuf buf;                 // storage
    DBuf op;                  // bf16 operand copy (BF16 mode)
    bool op_valid = false;
    DBuf op32;                // FP32 operand copy of FP64 storage (TF32 mode, FP32 refinement)
    bool op32_valid = false;
    bool valid = false;
    void rebind(cudaStream_t s) {
        buf.rebind(s);
        op.rebind(s);
        op32.rebind(s);
    }
    // The operand copies are rebuilt on demand (one flat copy each); dropping them between steps
    // keeps one storage copy per environment resident.
    void drop_operands() {
        op.release();
        op32.release();
        op_valid = op32_valid = false;
    }
    // An environment the sweep has moved past (it is rebuilt before it is read again).
    void release() {
        drop_operands();
        buf.release();
        valid = false;
    }
};

// ------------------------------------------------------------------------------------------
// Plans
// ------------------------------------------------------------------------------------------
struct TwoSiteMPO {            // nonzeros of sum_{w1} W1[w,s1,s1',w1] W2[w1,s2,s2',w2]
    struct E { int w, s1, s1p, s2, s2p, w2; double v; };
    std::vector<E> nz;
    int D0 = 0, D2 = 0, d = 0;
    std::vector<int> f0, f2;
};
TwoSiteMPO two_site_mpo(const SiteMPO& a, const SiteMPO& b);

struct HeffPlan {
    int prec = DMRG_FP64;
    PsiLayout psi;
    const EnvLayout* L = nullptr;
    const EnvLayout* R = nullptr;
    int ld_psi = 0, ld_y = 0;
    long long psiT_rows = 0, y_rows = 0, x_size = 0;
    CopyList pack;            // canonical x -> psiT slab
    CopyList unpack;          // FP32 result -> FP64 (accurate refinement plan)
    GemmBatch lstage, ldirect, rstage;   // L stage into X / straight into Y, R stage
    MixList mix;              // X -> Y slab
    std::vector<DiagJob> djobs;
    std::vector<DiagTerm> dterms;
    DBuf ddj, ddt, ddc;
    int diag_max = 0, diag_chunks = 0;
    double flops = 0.0;
    // scratch
    DBuf psiT, X, Y;
};
std::unique_ptr<HeffPlan> make_heff_plan(const Sec& bl, const Sec& br, const std::vector<int>& qn,
                                         const TwoSiteMPO& w12, const EnvLayout& L, const EnvLayout& R,
                                         int prec, cudaStream_t st);
void heff_apply(HeffPlan& P, const EnvSlab& L, const EnvSlab& R, const double* x, double* y,
                unsigned* err, cudaStream_t st);
void heff_diag(HeffPlan& P, const EnvSlab& L, const EnvSlab& R, double* out, cudaStream_t st);

// Left / right environment update through one site.
void env_update_left(const Sec& ba, const Sec& bb, const std::vector<int>& qn, const SiteMPO& W,
                     const EnvSlab& Lin, const double* A, EnvSlab& Lout, int prec, unsigned* err,
                     cudaStream_t st);
void env_update_right(const Sec& ba, const Sec& bc, const std::vector<int>& qn, const SiteMPO& W,
                      const EnvSlab& Rin, const double* B, EnvSlab& Rout, int prec, unsigned* err,
                      cudaStream_t st);
// Make sure the slab has storage for the layout and is zeroed.
void env_alloc(EnvSlab& e, const Sec& b, const std::vector<int>& flux, int prec, cudaStream_t st);
void env_make_operand(EnvSlab& e, int prec, cudaStream_t st);
// Packed canonical <-> slab conversions (FP64 packed on the device).
void env_from_packed(EnvSlab& e, const double* packed, cudaStream_t st);
void env_to_packed(const EnvSlab& e, double* packed, cudaStream_t st);
// The trivial boundary environment (one 1x1 block, value 1).
void env_boundary(EnvSlab& e, const Sec& b, const std::vector<int>& flux, int prec, cudaStream_t st);

// Two-site wavefunction from two packed site tensors: psi = left[(i,s1)] right[(m,s2)],
// optionally with the middle bond scaled by `mid` (per middle sector, FP64 device vector in
// sector order) -- used for the merge Psi' = psi_3 V psi_4.
void form_two_site(const Sec& bl, const Sec& bm, const Sec& br, const std::vector<int>& qn,
                   const double* left, const double* right, const double* mid, double* psi,
                   cudaStream_t st);

// Backward of the FP64 H_eff application on packed operands (L, R packed environments of the
// bonds bl / br for the MPO fluxes of w1 / w2): xbar, Lbar, Rbar (device) and W1bar, W2bar (dense
// host arrays, nullable) for ybar = dPhi/dy.  Synchronises the stream.
void heff_backward(const Sec& bl, const Sec& br, const std::vector<int>& qn, const SiteMPO& w1, const SiteMPO& w2,
                   const double* L_dev, const double* R_dev, const double* x_dev, const double* ybar_dev,
                   double* xbar_dev, double* Lbar_dev, double* Rbar_dev, double* W1bar, double* W2bar,
                   cudaStream_t st);

// SVD split of a packed two-site wavefunction.
struct SplitResult {
    Sec mid;                      // kept sectors of the new middle bond
    std::vector<double> lam;      // kept lambda (normalised), sector order, descending inside
    double trunc = 0.0;
    int sweeps = 0;               // Jacobi sweeps run
    int max_rows = 0;             // largest sector row count
};
// lam_pow_left/right: 0 or 1 -> A (left factor) multiplied by Lambda^pow_left, B by Lambda^pow_right.
SplitResult svd_split(const Sec& bl, const Sec& br, const std::vector<int>& qn1, const std::vector<int>& qn2,
                      const double* psi, int m_max, double rel_cutoff, bool accurate, int lam_pow_left,
                      int lam_pow_right, double* A_out, double* B_out, double* lam_out_dev, cudaStream_t st,
                      bool fp32 = false);
// One bond's split inside svd_split_batch (same meaning as svd_split's arguments).
struct SplitReq {
    Sec bl, br;
    const std::vector<int>* qn1 = nullptr;
    const std::vector<int>* qn2 = nullptr;
    const double* psi = nullptr;
    int m_max = 0;
    double rel_cutoff = 1e-12;
    int lam_pow_left = 0, lam_pow_right = 0;
    double* A_out = nullptr;
    double* B_out = nullptr;
    double* lam_out_dev = nullptr;
};
// The splits of several bonds in one pass: the charge sectors of all bonds form one batch of the
// Jacobi SVD (one cooperative launch), truncation (each bond's own keep-m rule), scatter and
// lambda then run per bond.  All psi must be ready on st; the outputs are written on st.
std::vector<SplitResult> svd_split_batch(const std::vector<SplitReq>& reqs, bool accurate, bool fp32,
                                         cudaStream_t st);
// FP64 re-orthonormalisation of the kept factor after a reduced-precision SVD: one Newton-Schulz
// step per middle sector, X <- X (3I - X^T X)/2 for a left factor (blocks bl x br, kept index on
// br), X <- (3I - X X^T)/2 X for a right factor (kept index on bl).
void orthonormalize_factor(const Sec& bl, const Sec& br, const std::vector<int>& qn, double* X, bool left,
                           cudaStream_t st);
// Flat element-type conversion of n elements (FP64 or FP32 source), stream-ordered.
void convert_flat(const void* src, Num in, void* dst, Num out, long long n, cudaStream_t st);
// Newton-Schulz orthonormalisation in FP64 of the square n x n matrices at v_off (column-major) of
// V, one per sector of ss, until |V^T V - I|_max < 1e-14.
void orthonormalize_square(const std::vector<SvdSec>& ss, double* V, cudaStream_t st);
// Worst-case (untruncated) element counts of the split's A and B outputs.
void svd_split_bounds(const Sec& bl, const Sec& br, const std::vector<int>& qn1, const std::vector<int>& qn2,
                      long long* a_elems, long long* b_elems, long long* lam_elems);

// Householder QR preconditioning of the one-sided Jacobi SVD (qr.cu).  Per sector: W (p x n,
// column-major at w_off, n <= p) and npanel T factors at t_off.
struct QrSec {
    long long w_off, t_off;
    int p, n;
};
// Largest sector row count whose QR panel fits in shared memory.
int qr_max_rows(bool f64);
struct QrPlan {
    std::vector<QrSec> secs;
    std::vector<int> act_off, trail_off, all_off;
    DBuf dsecs, dact, dtrail, dall, dcols, dxoff, dT;
    int npanel = 0, ncols = 0, max_rows = 0;
    bool ok = false;                  // false: a sector is too tall (use the plain Jacobi)
    // Lists for the sectors ss (w_off, p, n; v_off = offset of the n x n matrices X, V_J, Y).
    template <class T> void build(const std::vector<SvdSec>& ss, cudaStream_t st);
    // W <- R (on and above the diagonal) and the Householder vectors (below it).
    template <class T> void factor(T* W, cudaStream_t st);
    // X = R^T (n x n per sector at v_off).
    template <class T> void form_rt(const T* W, T* X, cudaStream_t st);
    // After the Jacobi on X (X V_J = Y): Y <- Y Sigma^-1 (the right singular vectors of W), Wout <-
    // Q [V_J Sigma; 0] (left singular vectors times Sigma), with the reflectors in W.
    template <class T> void finish(const T* W, T* Y, const T* VJ, T* Wout, cudaStream_t st);
};
// QR preconditioning of the split's Jacobi SVDs (on by default; the plain Jacobi when 0), set on
// the calling thread.
extern thread_local int g_svd_qr;

// Davidson on the projected Hamiltonian (FP64 vectors).
struct DavResult {
    double theta = 0.0, rnorm = 0.0;
    int iters = 0, matvecs = 0, acc_matvecs = 0;
    float mv_ms = 0.0f, acc_ms = 0.0f;
};
// Davidson with the plan's matvec; with `acc` (mixed modes) the run continues, restarted from the
// Ritz vector, for up to refine_iters iterations with the accurate matvec of `acc`.
DavResult davidson(HeffPlan& P, const EnvSlab& L, const EnvSlab& R, double* x, int kmax, double tol,
                   int max_iter, unsigned* err, cudaStream_t st, HeffPlan* acc = nullptr, int refine_iters = 0);

// Inverse canonical MPS gauge (Sec. IV): psi_j = Lambda_j Gamma_j Lambda_{j+1} on every site,
// V_b = Lambda_b^-1 on every inner bond, all site tensors in one FP64 slab.  Built from packed
// site tensors (bonds[0..L]) of a mixed-canonical state with its centre at `oc`; synchronises.
struct ICMPS;
ICMPS* icmps_build(const std::vector<Sec>& bonds, const std::vector<const double*>& sites, int oc,
                   const std::vector<int>& qn, cudaStream_t st);
void icmps_free(ICMPS* p);
const Sec& icmps_bond(const ICMPS& ic, int b);
const std::vector<double>& icmps_lambda(const ICMPS& ic, int b);
long long icmps_site_size(const ICMPS& ic, int j);
const double* icmps_site_dev(const ICMPS& ic, int j);
// One- and two-site expectation values over every site and every nearest-neighbour bond:
// ops1 [n1][d][d], ops2 [n2][d*d][d*d] (host, row index s1*d + s2), out1 [n1][L], out2 [n2][L-1]
// (host).  ms_out (nullable): device time of the measurement launches.  The host lists and
// buffers of a pass are kept in the gauge object for the next pass.  Synchronises.
void icmps_expectations(ICMPS& ic, const std::vector<int>& qn, int n1, const double* ops1, double* out1, int n2,
                        const double* ops2, double* out2, float* ms_out, cudaStream_t st);

// Scale the blocks of a packed site tensor (bonds bl x br) by a per-sector vector `lam` of
// the right bond (right_index = true: out[a][t] = in[a][t] lam[t]) or of the left bond
// (right_index = false: out[t][c] = lam[t] in[t][c]).
void scale_site(const Sec& bl, const Sec& br, const std::vector<int>& qn, const double* in, const double* lam,
                bool right_index, double* out, cudaStream_t st);
// Scale rows / columns of packed blocks (merge V, normalisation).
void scale_vec(double* x, long long n, double s, cudaStream_t st);
double dot_host(const double* x, const double* y, long long n, cudaStream_t st);

}  // namespace pd
