/*
 * pdmrg.h -- C ABI of the GB300 two-site DMRG engine (libpdmrg.so).
 *
 * The engine implements the serial two-site DMRG step and the real-space parallel scheme of
 * Stoudenmire & White, "Real-Space Parallel Density Matrix Renormalization Group":
 *   - the wavefunction on a bond, Sec. II Eq. (wf), optimised by Davidson with the
 *     Hamiltonian projected into the |a>|s1>|s2>|c> basis (Sec. II);
 *   - the SVD Psi = A Lambda B with truncation to the m largest singular values, Sec. II
 *     Eq. (svd), followed by the gauge move (A Lambda or Lambda B) and the transformation of
 *     the projected operators (Sec. II, operator-transformation paragraph);
 *   - the Lambda V Lambda split with V = Lambda^{-1} (Eqs. inverse, isvd), the merge
 *     Psi' = psi'_3 V psi'_4 (Eq. merge), the staggered sweep of Fig. 4, and the accurate
 *     recursive SVD of the Appendix at shared bonds.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  * Charges are integers (2*S^z, or all zero for a model without U(1) symmetry).  A bond is a
 *    list of sectors (q, m) with strictly ascending q.
 *  * MPO tensor W_j: row-major [D_j][d][d][D_{j+1}], W_j[w][s][s'][w'] = <s|op|s'>; every MPO
 *    channel w carries a flux f(w) and W_j[w][s][s'][w'] != 0 requires
 *    qn[s] - qn[s'] = f(w') - f(w).
 *  * Packed block layouts (all FP64, row-major inside a block, blocks back to back):
 *      site tensor  blocks (left sector i, local state s), i ascending then s ascending,
 *                   present when q_i + qn[s] is a sector of the right bond; block [m_i][m_r].
 *      two-site psi blocks (i, s1, s2) in that lexicographic order, present when
 *                   q_i + qn[s1] + qn[s2] is a sector of the right bond; block [m_i][m_c].
 *      environment  blocks (bra sector i, MPO channel w), i then w ascending, present when
 *                   q_i - f(w) is a sector of the same bond; block [m_i][m_ket].  Left
 *                   environments hold the projected operators of the left block (sites
 *                   0..j-1), right ones those of the right block.
 *  * Every function returns a dmrg_status and never aborts, throws or traps.  Device-side
 *    failures (capacity, non-finite values, a bounded wait that ran out) are recorded in a
 *    device error word and returned by the call that observes them.
 *  * Pointers named *_dev are device pointers owned by the caller; *_host are host pointers
 *    owned by the caller.  Inputs are read, never retained after the call returns.
 *  * `stream` arguments are cudaStream_t values (NULL = legacy default stream); calls are
 *    stream-ordered and return after the work is enqueued unless stated otherwise.
 */
#ifndef PDMRG_H
#define PDMRG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DMRG_OK = 0,
    DMRG_ERR_ARG = 1,       /* invalid argument (null pointer, bad size, inconsistent charges) */
    DMRG_ERR_CUDA = 2,      /* a CUDA runtime call failed; see dmrg_last_error */
    DMRG_ERR_OOM = 3,       /* device allocation failed */
    DMRG_ERR_CAPACITY = 4,  /* a size exceeds a fixed capacity of the engine */
    DMRG_ERR_QN = 5,        /* quantum-number bookkeeping inconsistency */
    DMRG_ERR_NUMERIC = 6,   /* non-finite value or breakdown detected */
    DMRG_ERR_TIMEOUT = 7,   /* a bounded device wait ran out (the kernel returned early) */
    DMRG_ERR_STATE = 8      /* call not valid in the context's current state */
} dmrg_status;

/* Arithmetic of the large contractions (H_eff matvec and environment updates).  The
 * Davidson Rayleigh-Ritz problem, re-orthogonalisation, SVD and Lambda^{-1} are FP64 in
 * every mode. */
typedef enum {
    DMRG_FP64 = 0,          /* FP64 everywhere (parity mode)                                   */
    DMRG_TF32 = 1,          /* tcgen05 kind::tf32, FP32 accumulate                             */
    DMRG_BF16 = 2           /* tcgen05 kind::f16 (bf16 operands), FP32 accumulate              */
} dmrg_precision;

/* ------------------------------------------------------------------------------------------
 * Problem description
 * ---------------------------------------------------------------------------------------- */
typedef struct {
    int n_sites;            /* L >= 2                                                         */
    int d;                  /* local dimension, 2..4                                          */
    const int* qn_local;    /* [d] charges of the local basis states                          */
    const int* D;           /* [L+1] MPO bond dimensions, D[0] = D[L] = 1                     */
    const int* flux;        /* [sum D] channel fluxes, bond 0 first                           */
    const double* W;        /* concatenated W_j, j = 0..L-1, row-major [D_j][d][d][D_{j+1}]    */
    int qn_total;           /* total charge of the state                                      */
} dmrg_mpo_desc;

typedef struct {
    const int* n_sectors;   /* [L+1] sectors per bond (bond 0 = {0}, bond L = {qn_total})      */
    const int* sector_q;    /* concatenated sector charges, bond 0 first                      */
    const int* sector_m;    /* concatenated sector dimensions                                 */
    const double* data;     /* concatenated packed site tensors, site 0 first                 */
    int canonical;          /* 0: arbitrary MPS, canonicalised by the engine (centre on site 0);
                               1: already mixed-canonical -- sites < center left-orthonormal,
                               sites > center right-orthonormal, normalised; no SVDs are run   */
    int center;             /* orthogonality centre when canonical = 1                        */
} dmrg_mps_desc;

typedef struct {
    int precision;          /* dmrg_precision                                                 */
    int kmax;               /* Davidson subspace size before restart (2..32, default 8)       */
    void* stream;           /* cudaStream_t base stream (region streams are forked from it)   */
    int svd_fp64;           /* mixed modes: 1 = ordinary-bond splits in FP64 as well (slower;
                               0 = FP32 block Jacobi + FP64 re-orthonormalisation)             */
    int fp64_emulation;     /* 1 = the context's FP64 grouped GEMMs (FP64-mode matvec and
                               environment updates, wavefunction formation, gauge moves, local
                               measurements) run FP64-accurate on the bf16 tensor cores
                               (dmrg_gemm64 mode 1); batches outside its K limit stay on the
                               FP64 units.  0 = FP64 units throughout.                          */
    int svd_plain_jacobi;   /* 1 = every split's one-sided Jacobi runs on the sector matrix W
                               itself; 0 (default) = on R^T from a Householder QR W = QR (a
                               few sweeps instead of many; sectors taller than the QR panel's
                               shared-memory limit, about 1700 rows, fall back to the plain
                               Jacobi)                                                          */
    int env_fp64;           /* mixed modes: 1 = environments stored and updated FP64-accurately
                               (FP64 GEMMs, on the tensor cores when fp64_emulation = 1; the
                               matvec reads bf16 / FP32 copies), so their rounding does not
                               compound from site to site; 0 (default) = FP32 storage and FP32
                               updates.  FP64 mode: no effect.                                  */
    int accurate_edges;     /* mixed modes: 1 = the region steps on the bonds next to a boundary
                               (those that produce and consume the edge tensors psi_3, psi_4 of
                               Eq. (merge)) and the merges themselves run Davidson in FP64 (FP64
                               matvec on FP64 copies of the environments, to a 1e-10 relative
                               residual, at most max(12, dav_max_iter + refine_iters)
                               iterations; counted as refinement matvecs); 2 = the same and FP64
                               splits at those steps; 0 (default) = the mixed-precision solve
                               everywhere.                                                     */
} dmrg_config;

typedef struct {
    int m_max;              /* kept states per bond (truncation target m)                     */
    double dav_tol;         /* Davidson stops when |r| <= dav_tol * max(1, |theta|)           */
    int dav_max_iter;       /* Davidson iteration cap per bond (tensor-core matvec in the
                               mixed modes)                                                   */
    int refine_iters;       /* mixed modes only: Davidson iterations continued from the Ritz
                               vector with an FP32-accurate matvec (0 = none)                 */
    int serial_regions;     /* region mode: 0 = one host thread and stream per region, the
                               regions' work overlapping on the GPU; 1 = the calling thread
                               runs the regions one after another (each gets the whole GPU;
                               the same results, since regions are independent between
                               merges); 2 = lockstep: the calling thread takes every region's
                               t-th bond step together -- Davidson region by region, then the
                               FP32 splits of all regions as one batch (one grouped Jacobi
                               launch, as dmrg_svd_split_batch), then each region's gauge move
                               and environment update; the results of 1 up to the rounding
                               of the FP32 splits                                             */
} dmrg_sweep_params;

typedef struct {
    double energy;          /* Davidson energy of the sweep's last local problem (last merge
                               with regions)                                                  */
    double max_trunc_err;   /* largest discarded weight of the sweep                          */
    int max_m;              /* largest bond dimension after truncation                        */
    int n_matvec;           /* H_eff applications                                             */
    int n_steps;            /* two-site steps (merges included)                               */
    int dav_nonconv;        /* local problems that hit dav_max_iter                           */
    double seconds;         /* host wall time of the call (synchronised)                      */
    double matvec_seconds;  /* summed device time of the matvecs (CUDA events)                */
    double matvec_flops;    /* algorithmic flops of those matvecs (nonzero blocks only)       */
    double min_fidelity;    /* smallest merge fidelity 1-|<Psi'|Psi>| of the sweep (-1: none;
                               an exact prediction can round a few ulps below 0)              */
    double max_fidelity;    /* largest merge fidelity of the sweep (-1: none)                 */
    int n_refine_matvec;    /* FP32-accurate refinement matvecs (mixed modes)                 */
    double refine_seconds;  /* their summed device time                                       */
} dmrg_sweep_stats;

typedef struct dmrg_ctx dmrg_ctx;

/* ------------------------------------------------------------------------------------------
 * Context API
 * ---------------------------------------------------------------------------------------- */

/* Create a context for the Hamiltonian given as an MPO (the "projected operators" of Sec. II
 * are built from it).  Copies the MPO to the device.  *out receives a context owned by the
 * caller and released with dmrg_destroy.  Errors: DMRG_ERR_ARG on inconsistent sizes or a
 * W entry that violates the flux rule. */
dmrg_status dmrg_init_mpo(dmrg_ctx** out, const dmrg_mpo_desc* mpo, const dmrg_config* cfg);

/* Load a matrix product state (packed layout above, host memory, copied).  With canonical = 0
 * the engine brings it to right-canonical form with the orthogonality centre on site 0 by
 * untruncated SVDs from the right and normalises it; with canonical = 1 it trusts the given
 * mixed-canonical gauge.  Then every environment on both sides of the centre is built.
 * Serial mode afterwards. */
dmrg_status dmrg_set_mps(dmrg_ctx* ctx, const dmrg_mps_desc* mps);

/* Serial mode: n two-site steps continuing the current sweep (moving right until the centre
 * reaches site L-1, then left until site 0, and so on).  2(L-1) steps from site 0 are one
 * sweep.  Blocks until done; stats (nullable) cover these steps. */
dmrg_status dmrg_advance(dmrg_ctx* ctx, int n_steps, const dmrg_sweep_params* p, dmrg_sweep_stats* stats);

/* Real-space parallel set-up (Sec. II, Fig. 4): split the chain into n_regions blocks at
 * bonds round(k L / n_regions); run `warmup` serial sweeps (the last one's left half-sweep
 * performs the Lambda V Lambda split at every boundary it crosses; warmup = 0 moves the
 * gauge by untruncated SVDs instead), then move even regions (1-based) to their right end.
 * Each region gets its own CUDA stream.  n_regions = 1 returns to serial mode. */
dmrg_status dmrg_setup_regions(dmrg_ctx* ctx, int n_regions, int warmup,
                               const dmrg_sweep_params* p);

/* One sweep.  Serial mode: bonds 0..L-2 moving right, then L-2..0 moving left.  Region mode:
 * Fig. 4 (a)-(d) with every region on its own stream, merges (Eq. merge) at the meeting
 * boundaries after both regions arrived.  Blocks until the sweep is done.  stats may be NULL. */
dmrg_status dmrg_sweep(dmrg_ctx* ctx, const dmrg_sweep_params* p, dmrg_sweep_stats* stats);

/* Merge at region boundary k (1..n_regions-1): Psi' = psi'_3 V psi'_4 with the stored V
 * (Eq. merge), normalisation, Davidson on the shared bond with the left environment of the
 * left region and the right environment of the right region, accurate SVD (Appendix),
 * new V = Lambda^{-1}, environment hand-off.  Both regions must sit at the boundary.
 * fidelity_out (nullable) receives 1 - |<Psi'|Psi>|; energy_out (nullable) the energy. */
dmrg_status dmrg_merge(dmrg_ctx* ctx, int k, const dmrg_sweep_params* p,
                       double* fidelity_out, double* energy_out);

/* FP64 Rayleigh quotient <psi|H_eff|psi>/<psi|psi> of the current two-site wavefunction
 * (serial mode) -- the energy of the whole state when the environments are current.  Mixed
 * modes keep the environments in FP32, whose rounding (compounded over the sites) biases this
 * value: ~3e-5 relative on the 24x8 Heisenberg cylinder at m = 300, while the state itself is
 * within 1e-5 of the FP64 path's.  The exact energy of a mixed-mode state: export it
 * (dmrg_get_site, dmrg_get_bond, dmrg_get_center) into an FP64 context and call this there. */
dmrg_status dmrg_energy(dmrg_ctx* ctx, double* E_out);

/* Sector table of bond b (0..L): writes up to cap entries, *n_out = number of sectors.
 * In region mode the bond is read from the region that owns it. */
dmrg_status dmrg_get_bond(dmrg_ctx* ctx, int b, int* q_out, int* m_out, int cap, int* n_out);

/* Singular values stored for bond b by its last SVD (descending within each sector,
 * sectors ascending, normalised to sum lambda^2 = 1).  *n_out = count. */
dmrg_status dmrg_get_lambda(dmrg_ctx* ctx, int b, double* lam_out, int cap, int* n_out);

/* Gradient of the energy E = <Psi|H|Psi>/<Psi|Psi> of the serial state with respect to every
 * MPO tensor (FP64 contexts; no counterpart in the paper): Wbar (host, caller owned) receives the
 * tensors dE/dW_j in the layout of dmrg_mpo_desc.W (site after site, [D_j][d][d][D_{j+1}]),
 * exact at the nonzero entries of the MPO and zero elsewhere.  For a variationally optimised
 * state, dE/dtheta = sum_j <Wbar_j, dW_j/dtheta> for any MPO parameter theta (Hellmann-Feynman).
 * One gauge sweep: at each bond the backward of the projected Hamiltonian with ybar = psi gives
 * the gradient of the left site (the last bond also the right one); the centre is moved by
 * untruncated SVDs and returned to site 0.  E_out (nullable): <psi|H_eff|psi> at the last bond.
 * Region mode or mixed precision: DMRG_ERR_STATE. */
dmrg_status dmrg_energy_gradient(dmrg_ctx* ctx, double* Wbar, double* E_out);

/* Site tensor j of the state (checkpointing): the packed layout of dmrg_set_mps for bonds
 * (j, j + 1) as dmrg_get_bond reports them, copied to host memory out[cap] (FP64, caller owned);
 * *n_out = its element count (DMRG_ERR_CAPACITY, with *n_out set, if cap is smaller).  Serial
 * mode: together with dmrg_get_bond and dmrg_get_center this reproduces the state through
 * dmrg_set_mps (canonical = 1).  Region mode: site j of the region holding it, except that the
 * first site of every region right of a boundary b carries V_b = Lambda_b^-1 on its left bond, so
 * the exported sites contract to the real-space parallel state, the regions joined by V at every
 * boundary as in Eq. (merge); that MPS is not canonical (load it with canonical = 0).
 * Synchronises the stream. */
dmrg_status dmrg_get_site(dmrg_ctx* ctx, int j, double* out, long long cap, long long* n_out);

/* Inverse canonical gauge of the serial state (Sec. IV, Figs. 8 and 9): a copy of the state,
 * kept in the context, in which every site tensor psi_j = Lambda_j Gamma_j Lambda_{j+1} is an
 * orthogonality centre and every inner bond b (joining sites b-1 and b) carries the diagonal
 * V_b = Lambda_b^{-1} of inverse Schmidt weights: |Psi> = psi_0 V_1 psi_1 ... V_{L-1} psi_{L-1}.
 * Built in FP64 (any precision mode) by untruncated SVDs: the centre is moved to site 0, then
 * Fig. 8's step (SVD, one copy of Lambda into each neighbour, V on the bond) is taken at every
 * bond left to right; Schmidt values at or below 1e-12 of the largest are dropped so that V is
 * finite.  The engine's own state is not changed; a later set_mps, sweep, advance, region set-up
 * or merge discards the copy.  Region mode: DMRG_ERR_STATE.  Synchronises the stream. */
dmrg_status dmrg_inverse_canonical(dmrg_ctx* ctx);

/* Sectors of bond b (0..L) of the inverse canonical copy (as dmrg_get_bond). */
dmrg_status dmrg_icmps_bond(dmrg_ctx* ctx, int b, int* q_out, int* m_out, int cap, int* n_out);

/* V_b = 1/Lambda_b of the inverse canonical copy in the sector order of dmrg_icmps_bond
 * (ascending within each sector; bonds 0 and L: the single value 1). */
dmrg_status dmrg_icmps_v(dmrg_ctx* ctx, int b, double* v_out, int cap, int* n_out);

/* Site tensor psi_j of the inverse canonical copy (packed layout of dmrg_set_mps for the bonds
 * of dmrg_icmps_bond), copied to host memory out[cap]; *n_out = element count
 * (DMRG_ERR_CAPACITY, with *n_out set, if cap is smaller).  Synchronises the stream. */
dmrg_status dmrg_icmps_site(dmrg_ctx* ctx, int j, double* out, long long cap, long long* n_out);

/* Local expectation values in the inverse canonical gauge (Sec. IV): as every psi_j is an
 * orthogonality centre, <O_j> = <psi_j|O|psi_j>/<psi_j|psi_j> and a nearest-neighbour operator
 * needs only Theta_j = psi_j V_{j+1} psi_{j+1}: <O_{j,j+1}> = <Theta_j|O|Theta_j>/<Theta_j|Theta_j>.
 * Every site and every bond is measured in one pass (a column scaling, one grouped GEMM forming
 * all Theta_j, one launch of block dot products, a fixed-order reduction, one contraction per
 * operator set).  ops1: n_ops1 one-site operators [d][d] (row s, column s'); ops2: n_ops2
 * two-site operators [d*d][d*d] (row index s1*d + s2); both host, real, caller owned.  Only the
 * matrix elements between basis states of equal total charge contribute (others vanish in a U(1)
 * eigenstate).  out1 [n_ops1][L] and out2 [n_ops2][L-1] (host, caller owned; nullable when the
 * count is 0).  ms_out (nullable): device time of the measurement launches in ms.  Needs
 * dmrg_inverse_canonical first (else DMRG_ERR_STATE).  Synchronises the stream. */
dmrg_status dmrg_local_expectations(dmrg_ctx* ctx, int n_ops1, const double* ops1, double* out1,
                                    int n_ops2, const double* ops2, double* out2, float* ms_out);

/* Orthogonality-centre site of the serial state, or of region k in region mode. */
dmrg_status dmrg_get_center(dmrg_ctx* ctx, int region, int* site_out);

dmrg_status dmrg_destroy(dmrg_ctx* ctx);

/* Message of the last failure on this context (context-owned, valid until the next call). */
const char* dmrg_last_error(const dmrg_ctx* ctx);
const char* dmrg_status_string(int status);

/* ------------------------------------------------------------------------------------------
 * Instrumentation (process-wide).  Kernel launches are always counted; with profiling on, the
 * grouped-GEMM launches are bracketed by CUDA events on their own stream and their device
 * time and algorithmic flops are accumulated per class.  Environment updates run at FP32
 * accuracy or better in every mode (their rounding errors compound from site to site), so in
 * the mixed modes they appear under f32_gemm_*.
 * ---------------------------------------------------------------------------------------- */
typedef struct {
    long long launches;          /* kernels launched by the library since the last reset       */
    long long mv_gemm_launches;  /* tensor-core GEMM launches of H_eff matvecs                  */
    double mv_gemm_ms;           /* their summed device time                                    */
    double mv_gemm_flops;        /* their algorithmic flops                                     */
    long long env_gemm_launches; /* GEMM batches of environment updates: tensor core, and FP64
                                    (emulated or FP64 units) with FP64-accurate environments   */
    double env_gemm_ms;
    double env_gemm_flops;
    long long f64_gemm_launches; /* FP64 grouped-GEMM launches (any use)                        */
    double f64_gemm_ms;
    double f64_gemm_flops;
    long long f32_gemm_launches; /* FP32 SIMT grouped-GEMM launches (mixed-mode environments)   */
    double f32_gemm_ms;
    double f32_gemm_flops;
    long long svd_calls;         /* block-sparse SVD passes (one per split, or one per batch of
                                    splits of several regions' bonds run together)               */
    long long svd_sweeps;        /* Jacobi sweeps they ran in total                             */
    double svd_ms;               /* device time of their Jacobi kernels                         */
    long long svd_block_calls;   /* of those, FP32 splits run by the block Jacobi                */
    long long svd_fp64_calls;    /* of those, FP64 splits (parity mode, shared bonds)            */
    double svd_block_ms;         /* device time of the block-Jacobi splits                      */
    double svd_fp64_ms;          /* device time of the FP64 splits                              */
    long long svd_max_rows;      /* largest sector row count seen                               */
    long long svd_fp64_fallbacks; /* FP32 splits redone in FP64 (re-orthonormalisation refused)  */
    double svd_block_flops;      /* FP32 Gram + column-rotation flops of the block-Jacobi splits */
    long long svd_rot_hist[48];  /* block Jacobi: block pairs rotated in sweep i, summed over splits */
    long long emu_fallbacks;     /* emulated FP64 GEMM batches sent to the FP64 units by the scale
                                    guard (a shared operand row's scale class far above a problem's
                                    own row maximum) or by a NaN/Inf operand                     */
    long long tune_classes;      /* tensor-core GEMM shape classes whose tile width was chosen by
                                    timing every width (process-wide, not reset)               */
    long long tune_changed;      /* of those, classes where the timing overruled the cost model  */
    long long svd_bonds;         /* bonds split by those passes                                   */
    double svd_block_alg_flops;  /* FP32 splits: textbook SVD flops of their sector matrices, the
                                    R-SVD with U and V, 4 p n^2 + 22 n^3 per p x n sector         */
    double svd_block_alg_bytes;  /* FP32 splits: the sector matrices read once, U and V written
                                    once (FP32), 4 (2 p n + n^2) per sector                      */
} dmrg_profile;

void dmrg_profile_enable(int on);
void dmrg_profile_reset(void);
/* Synchronises the device, then copies the counters. */
dmrg_status dmrg_profile_read(dmrg_profile* out);

/* Throughput probes (the library's own kernels, timed with CUDA events on `stream`), for roofline
 * denominators: kind 0 = FP64 FMA rate of the SMs (eight independent DFMA chains per thread),
 * 1 = FP32 FMA rate (the same with FFMA), 2 = this library's tcgen05 grouped GEMM on one dense
 * 8192^3 bf16 problem (FP32 accumulation), 3 = the same in tf32.  *tflops_out in TFLOP/s.  The
 * GEMM probes allocate about 0.8 GB for their operands while they run.  Kinds 2-3 without sm_103
 * tensor cores: DMRG_ERR_STATE.  Synchronises the stream.  No counterpart in the paper. */
dmrg_status dmrg_probe(int kind, double* tflops_out, void* stream);

/* ------------------------------------------------------------------------------------------
 * Operation API: single steps on caller-provided device buffers (used for element-wise
 * parity tests and micro-benchmarks).  Layouts are the packed layouts above.
 * ---------------------------------------------------------------------------------------- */
typedef struct {
    int d;
    const int* qn_local;    /* [d]                                                            */
    int nl; const int* ql; const int* ml;   /* bond left of site 1  (sectors of psi's a)       */
    int nr; const int* qr; const int* mr;   /* bond right of site 2 (sectors of psi's c)       */
    int D0, D1, D2;         /* MPO bonds around the two sites                                 */
    const int* f0; const int* f1; const int* f2;   /* their channel fluxes                    */
    const double* W1;       /* [D0][d][d][D1] host                                            */
    const double* W2;       /* [D1][d][d][D2] host                                            */
} dmrg_bond_desc;

/* y = H_eff x with H_eff = L x W1 x W2 x R (Sec. II projected Hamiltonian, written as
 * out[a',s1,s2,c'] = sum L[a',w,a] W1[w,s1,s1',w'] W2[w',s2,s2',w''] R[c',w'',c] x[a,s1',s2',c]).
 * L_dev, R_dev: packed environments of the left/right bond; x_dev, y_dev: packed two-site
 * vectors (FP64).  prec selects the contraction arithmetic.  flops_out (nullable) receives
 * the algorithmic flop count of one application. */
dmrg_status dmrg_heff_apply(const dmrg_bond_desc* bd, int prec, const double* L_dev,
                            const double* R_dev, const double* x_dev, double* y_dev,
                            double* flops_out, void* stream);

/* Same result as dmrg_heff_apply in FP64 (prec = DMRG_FP64), for callers that cannot allocate
 * device memory -- for example code whose device allocations are all owned by an external
 * memory manager, or a thread that must not enter the CUDA allocator.  It makes no device
 * allocation of any kind: the scratch it needs (job lists, the L-stage intermediate and the
 * MPO-mixed intermediate) lives in one fixed 64 MiB device array inside the library, which
 * every GPU that loads the library holds until the process exits.  The paper has no
 * counterpart of this entry point.
 *  - Inputs/outputs and layouts as in dmrg_heff_apply (device pointers owned by the caller).
 *  - The first call on a device, made with that device current, looks up the array's device
 *    address (cudaGetSymbolAddress) and caches it; make that first call before any stream
 *    capture.
 *  - All calls share the array and leave their intermediates in it; calls whose GPU work
 *    overlaps (different streams without ordering) race on it.
 *  - DMRG_ERR_CAPACITY when the bond needs more than the 64 MiB of scratch. */
dmrg_status dmrg_heff_apply_noalloc(const dmrg_bond_desc* bd, const double* L_dev, const double* R_dev,
                                    const double* x_dev, double* y_dev, void* stream);

/* Left-environment update through one site (Sec. II operator transformation by A):
 * Lout[b',w',b] = sum A[a',s,b'] Lin[a',w,a] W[w,s,s',w'] A[a,s',b].  Bonds: (nl,ql,ml) left
 * of the site, (nr,qr,mr) right of it; D0/f0 and D1/f1 the MPO bonds, W1 the site's MPO
 * tensor (D2, f2, W2 unused). */
dmrg_status dmrg_env_left(const dmrg_bond_desc* bd, int prec, const double* Lin_dev,
                          const double* A_dev, double* Lout_dev, void* stream);

/* Backward of the H_eff application (FP64; no counterpart in the paper, which has no
 * derivatives): given ybar = dPhi/dy for y = H_eff(L, W1, W2, R) x, the gradients
 *   xbar[a,s1',s2',c] = sum ybar[a',s1,s2,c'] L[a',w,a] W1[w,s1,s1',w'] W2[w',s2,s2',w''] R[c',w'',c]
 *   Lbar[a',w,a], Rbar[c',w'',c]  (packed environment layouts of the bond descriptor)
 *   W1bar[w,s1,s1',w'], W2bar[w',s2,s2',w''] (dense, host, nullable; exact at every nonzero entry
 *   of W1 / W2, zero elsewhere: the MPO's sparsity pattern is fixed)
 * x, ybar, xbar: packed two-site layout; L, R, Lbar, Rbar: packed environments (device, caller
 * owned, outputs overwritten).  The forward intermediates are recomputed from x.  Synchronises
 * the stream. */
dmrg_status dmrg_heff_backward(const dmrg_bond_desc* bd, const double* L_dev, const double* R_dev,
                               const double* x_dev, const double* ybar_dev, double* xbar_dev,
                               double* Lbar_dev, double* Rbar_dev, double* W1bar, double* W2bar,
                               void* stream);

/* Right-environment update (operator transformation by B):
 * Rout[a',w,a] = sum B[a',s,c'] Rin[c',w',c] W[w,s,s',w'] B[a,s',c]. */
dmrg_status dmrg_env_right(const dmrg_bond_desc* bd, int prec, const double* Rin_dev,
                           const double* B_dev, double* Rout_dev, void* stream);

/* Two-site SVD with truncation (Eq. svd): psi (packed two-site) -> A (packed site tensor on
 * the left bond x new middle bond), lambda, B (packed site tensor middle x right).  The kept
 * set: lambda <= 1e-12 lambda_max dropped; order (lambda desc, q asc, index asc); first m_max
 * kept; a degenerate group at the cut (relative gap <= 1e-10) dropped whole.  lambda is
 * normalised to sum lambda^2 = 1.  `accurate` selects the mode: 0 FP64 one-sided Jacobi; 1 the
 * same with the Appendix recursion (eps 1e-4); 2 the mixed-precision engine's split: FP32 block
 * Jacobi, cutoff raised to 1e-5 lambda_max (above the FP32 rounding level), A re-orthonormalised
 * in FP64 (Newton-Schulz), B = V^T as computed in FP32.  Adding 4 to the mode runs the Jacobi
 * on the sector matrices themselves instead of on R^T from their Householder QR (the default
 * for modes 0-2).  Other values: DMRG_ERR_ARG.
 * Outputs: middle-bond sectors (nm_out, qm_out[cap], mm_out[cap]), A_dev/B_dev/lam_dev sized
 * by the caller for the worst case (no truncation), trunc_out (nullable) the discarded weight.
 * Synchronises the stream (the kept sector sizes are returned to the host). */
dmrg_status dmrg_svd_split(const dmrg_bond_desc* bd, const double* psi_dev, int m_max,
                           int accurate, double* A_dev, double* lam_dev, double* B_dev,
                           int cap, int* nm_out, int* qm_out, int* mm_out, double* trunc_out,
                           void* stream);

/* The two-site splits (Eq. svd) of n_bonds bonds in one pass -- the concurrent bond steps of the
 * real-space regions, Sec. II and Fig. 4: the charge sectors of all bonds form one batch of the
 * Jacobi SVD (one grouped launch, which fills the GPU where a single bond's few large sectors
 * leave most SMs idle), then truncation, lambda and the factors follow bond by bond, each bond
 * with its own keep-m rule.  Every bond's outputs are those dmrg_svd_split returns for it alone
 * in the same mode up to rounding: rotation thresholds are per sector, but how a sector's columns
 * are staged (and so the rounding of its rotations) depends on the batch's largest sector.  Host
 * arrays of n_bonds entries:
 * bds (descriptors), psi_devs, A_devs, lam_devs, B_devs (device buffers owned by the caller and
 * sized as for dmrg_svd_split), m_max; mode as for dmrg_svd_split (0-2, +4), the same for every
 * bond.  Outputs: nm_out[n_bonds]; qm_out, mm_out[n_bonds * cap] (bond b's sectors from b * cap);
 * trunc_out[n_bonds] (nullable).  n_bonds = 0 does nothing.  Synchronises the stream. */
dmrg_status dmrg_svd_split_batch(int n_bonds, const dmrg_bond_desc* bds, const double* const* psi_devs,
                                 const int* m_max, int mode, double* const* A_devs,
                                 double* const* lam_devs, double* const* B_devs, int cap, int* nm_out,
                                 int* qm_out, int* mm_out, double* trunc_out, void* stream);

/* One problem of a grouped FP64 GEMM:
 *   C(m, n) (+)= alpha * sum over its segments sum_{k < K} A(m, k) B(n, k),   m < M, n < N,
 *   A(m, k) = A[a_off + m*sam + k*sak], B(n, k) = B[b_off + n*sbn + k*sbk],
 *   C(m, n) = C[c_off + m*scm + n*scn];  accumulate = 0: C = ..., 1: C += ...
 * Segments seg0 .. seg0 + nseg - 1 of the segment array.  No two problems of one call may
 * write the same element of C.  (The block contractions of Sec. II -- projected Hamiltonian,
 * operator transformation, two-site wavefunction -- are all batches of this form.) */
typedef struct {
    int M, N, seg0, nseg;
    long long c_off;
    int sam, sak, sbn, sbk, scm, scn;
    int accumulate, pad_;
    double alpha;
} dmrg_gemm_problem;
typedef struct {
    long long a_off, b_off;
    int K, pad_;
} dmrg_gemm_segment;

/* Grouped FP64 GEMM on device buffers A_dev, B_dev, C_dev (caller owned; every addressed
 * element must lie inside them -- not checked).  mode 0: the FP64 units.  mode 1: FP64-accurate
 * emulation on the bf16 tensor cores (Ozaki, Ogita and Oishi's error-free splitting): each
 * operand row is scaled by a power of two and cut into s slices of beta bits, the slice
 * products are summed exactly in FP32 on the tensor cores and combined in FP64; the error is
 * below (s^2/2 + 2) 2^(-s beta) max_k|A(m,k)| max_k|B(n,k)| per term (s beta >= 56), at the level
 * of FP64 rounding.  Operand rows that several problems share get one scale, that of the largest
 * row they meet in any problem; when a problem's own row (column) maximum lies more than 3 bits
 * below that scale, or an operand is NaN or Inf, the whole batch runs on the FP64 units instead
 * (counted in dmrg_profile.emu_fallbacks).  info (nullable, int[3]): beta, s and the number of
 * FP32 accumulators per problem (0, 0, 0 in mode 0 and when the batch ran on the FP64 units).
 * Errors: DMRG_ERR_ARG (bad problem or segment), DMRG_ERR_STATE
 * (mode 1 without sm_103 tensor cores), DMRG_ERR_CAPACITY (mode 1 with a K too large for exact
 * FP32 accumulation, about 2 million per problem).  Synchronises the stream; an empty batch
 * returns DMRG_OK without any device call. */
dmrg_status dmrg_gemm64(const dmrg_gemm_problem* probs, int n_probs, const dmrg_gemm_segment* segs, int n_segs,
                        const double* A_dev, const double* B_dev, double* C_dev, int mode, int* info,
                        void* stream);

#ifdef __cplusplus
}
#endif
#endif /* PDMRG_H */
