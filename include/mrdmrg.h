/*
 * mrdmrg.h -- C ABI of the GB300 (sm_103a) hot path of two-site DMRG on a cylinder in
 * mixed real and momentum space (Motruk, Zaletel, Mong, Pollmann, arXiv:1512.03318).
 *
 * Problem statement (Sec. III.A, Eq. H; Sec. IV.D, Eqs. H_kin and H_k_int): spinless
 * fermions on an Lx x Ly cylinder (open along x, periodic around y) with hopping t, flux
 * phi = 2 pi p / q per plaquette in Landau gauge and nearest-neighbour repulsion V. The
 * orbitals around each ring are Fourier transformed, so the chain runs over orbitals
 * (x, k) with k = 2 pi m / Ly (Sec. II, Fig. 1b) and the rotation of the cylinder becomes
 * an onsite Z_Ly charge K next to the particle number N (Sec. II).
 *
 * Conventions shared by every call
 *   charge      (N, K) with K in [0, modulus); modulus = Ly in the mixed basis, 1 in real
 *               space. Local charge of an orbital with momentum index m and occupation s:
 *               q(s) = (s, s*m mod modulus).
 *   sectors     int32 triplets (N, K, dim), strictly increasing in (N, K), dim > 0.
 *   channels    MPO channel charges, int32 pairs (dN, dK); an MPO entry W[w, w', s', s]
 *               (s' bra, s ket) is allowed only if c_{w'} = c_w + q(s') - q(s).
 *   complex     interleaved (re, im) doubles (complex128); lengths below count complex
 *               elements.
 *   theta       two-site tensor, fused by middle charge q_m: for each q_m (sorted) a dense
 *               block with rows (s1, a), q_a + q1(s1) = q_m, s1 = 0 rows first, and columns
 *               (s2, b), q_b - q2(s2) = q_m, s2 = 0 first; row-major; blocks back to back.
 *   left env    L_w blocks for every (w, a) with q_a + c_w a left sector, shape
 *               d(q_a + c_w) x d(q_a) ([bra][ket]); ordered by w then a; row-major.
 *   right env   R_w blocks for every (w, b) with q_b + c_w a right sector, shape
 *               d(q_b) x d(q_b + c_w) ([ket][bra]); ordered by w then b; row-major.
 *   H_eff       theta'[a',s1',s2',b'] = sum L_w[a',a] W_i[w,w',s1',s1] W_{i+1}[w',w'',s2',s2]
 *               R_{w''}[b,b'] theta[a,s1,s2,b]  (the two-site effective Hamiltonian of
 *               DMRG; the paper relies on standard DMRG, its refs. W92, S2005, S2011).
 *
 * Pointers: "dev" arguments are device pointers on the context's device, owned by the
 * caller and only read or written during the call (or until the stream work it enqueued
 * completes). Host arrays are read during the call only. Handles are owned by the library
 * and released by the matching *_free. Every call returns 0 or a negative MRD_E_* code and
 * never aborts; mrd_last_error() gives a message. Calls on one context are not
 * thread-safe. All device work is enqueued on the context's stream.
 */
#ifndef MRDMRG_H
#define MRDMRG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MRD_OK 0
#define MRD_E_ARG (-1)      /* invalid argument (sizes, ordering, null pointer)           */
#define MRD_E_CHARGE (-2)   /* an MPO entry or block violates charge conservation          */
#define MRD_E_NOCONV (-3)   /* an iterative solver did not converge                       */
#define MRD_E_OOM (-4)      /* device allocation failed                                   */
#define MRD_E_CUDA (-5)     /* a CUDA runtime call failed                                 */
#define MRD_E_NAN (-6)      /* a non-finite value was produced                            */
#define MRD_E_TIMEOUT (-7)  /* a bounded device wait gave up                              */
#define MRD_E_STATE (-8)    /* call out of order (e.g. apply before set_env)              */
#define MRD_E_HOST (-9)     /* host memory or threads exhausted (no C++ exception leaves  */
                            /* the library; the handles of the failed call may be stale:  */
                            /* destroy them)                                              */

#define MRD_PREC_FP64 0     /* complex128 operands, FP64 arithmetic                       */
#define MRD_PREC_TF32 1     /* tcgen05 tensor cores, TF32 operands, FP32 accumulation     */
#define MRD_PREC_BF16X3 2   /* tcgen05, split BF16 (hi*hi + hi*lo + lo*hi), FP32 accum.   */
#define MRD_PREC_FF 3       /* complex128 operands split into float-float pairs (~48-bit  */
                            /* products, TwoSum accumulation) on the FP32 pipes           */

#define MRD_BASIS_MIXED 0   /* orbitals (x, k_m), charges (N, K mod Ly)                   */
#define MRD_BASIS_REAL 1    /* orbitals (x, y), charge N only (modulus 1)                 */
#define MRD_BASIS_MIXED_REAL 2 /* orbitals (x, k_m), charges (N, K mod Ly), the sine /     */
                               /* cosine machine of Sec. IV.D (Eq. rot): every entry real  */

typedef struct mrd_ctx mrd_ctx;
typedef struct mrd_mpo mrd_mpo;
typedef struct mrd_heff mrd_heff;
typedef struct mrd_dmrg mrd_dmrg;

/* ------------------------------------------------------------------ context */

/* Create a context on CUDA device `device`. `stream` is a cudaStream_t borrowed from the
 * caller (NULL = the legacy default stream); the library never destroys it. */
int mrd_create(mrd_ctx** out, int device, void* stream);
int mrd_destroy(mrd_ctx* ctx);
int mrd_set_stream(mrd_ctx* ctx, void* stream);
/* Return to the device the memory the library keeps cached for reuse on this context's device
 * (blocks released by freed handles); waits for the context stream first. Memory of live
 * handles is not touched. */
int mrd_release_cached(mrd_ctx* ctx);
/* Message of the last failing call on this context (static storage of the context). */
const char* mrd_last_error(const mrd_ctx* ctx);
/* Library version as major*10000 + minor*100 + patch. */
int mrd_version(void);
/* Number of CUDA kernels this library has launched so far in this process (all contexts). */
int64_t mrd_launch_count(void);

/* ------------------------------------------------------------------ MPO (Sec. IV) */

typedef struct {
  int32_t lx, ly;          /* rings along the cylinder, orbitals per ring (ly >= 2)      */
  int32_t flux_p, flux_q;  /* flux per plaquette phi = 2 pi p / q (q > 0)                */
  double t, v;             /* hopping and nearest-neighbour repulsion                    */
  int32_t basis;           /* MRD_BASIS_MIXED, MRD_BASIS_REAL or MRD_BASIS_MIXED_REAL    */
} mrd_model;

/* Build the Hamiltonian MPO from its finite-state machine (Sec. IV.A-B): intermediate
 * nodes carry the set of operators already placed and, in the mixed basis, the cumulative
 * momentum (the momentum-labelled nodes of Sec. IV.D, Figs. 9-10); unreachable nodes are
 * trimmed (Sec. IV.D) and nodes with proportional pasts or futures are fused. Host
 * computation; the result lives in host memory of the handle. ctx may be NULL (no device
 * is touched; errors are then reported by the return code only). */
int mrd_mpo_build(mrd_ctx* ctx, const mrd_model* model, mrd_mpo** out);
int mrd_mpo_free(mrd_mpo* mpo);
/* Number of sites (lx*ly) and charge modulus. */
int mrd_mpo_info(const mrd_mpo* mpo, int32_t* n_sites, int32_t* modulus);
/* Dimension of MPO bond `bond` (0..n_sites); if charges != NULL, writes 2*dim int32
 * (dN, dK) channel charges. */
int mrd_mpo_bond(const mrd_mpo* mpo, int32_t bond, int32_t* dim, int32_t* charges);
/* Nonzero entries of site `site`: if idx != NULL writes 4*nnz int32 (w, w', s', s) and if
 * val != NULL 2*nnz doubles (re, im), ordered by (w, w', s', s). */
int mrd_mpo_site(const mrd_mpo* mpo, int32_t site, int32_t* nnz, int32_t* idx, double* val);
/* MPO diagnostics of Sec. IV.D (its figure of the mean bond dimension <D> against the
 * circumference, and of the fraction of nonzero MPO entries), over the `count` sites
 * first .. first+count-1 (e.g. one ring, first = x*ly, count = ly) and the bonds
 * first .. first+count-1 to their left: out4 = {mean bond dimension, largest bond dimension,
 * mean fill (nonzero entries of site j / (D_j * D_{j+1} * 4)), total nonzero entries}.
 * MRD_E_ARG unless 0 <= first and 1 <= count and first + count <= n_sites. Host only. */
int mrd_mpo_stats(const mrd_mpo* mpo, int32_t first, int32_t count, double* out4);

/* ------------------------------------------------------------------ two-site H_eff */

typedef struct {
  int32_t n_left;  const int32_t* left;    /* sectors of the bond left of site i         */
  int32_t n_right; const int32_t* right;   /* sectors of the bond right of site i+1      */
  int32_t m1, m2, modulus;                 /* momentum indices of sites i, i+1; modulus  */
  int32_t d_l, d_m, d_r;                   /* MPO bond dims left of i, between, right    */
  const int32_t* c_l; const int32_t* c_m; const int32_t* c_r;   /* channel charges       */
  int32_t nnz_i; const int32_t* wi_idx; const double* wi_val;   /* W_i entries           */
  int32_t nnz_j; const int32_t* wj_idx; const double* wj_val;   /* W_{i+1} entries       */
} mrd_heff_desc;

/* Validate the description and build, on the device, the charge tables of the two-site
 * problem: fused middle sectors with block offsets, environment block layouts, and the
 * task lists of the contraction. Host arrays are copied. */
int mrd_heff_create(mrd_ctx* ctx, const mrd_heff_desc* desc, mrd_heff** out);
int mrd_heff_free(mrd_heff* h);
/* Lengths (complex elements) of theta, the left env and the right env. */
int mrd_heff_sizes(const mrd_heff* h, int64_t* theta_len, int64_t* lenv_len, int64_t* renv_len);
/* Load the environments (device pointers, complex128, layouts above). They are folded
 * with the MPO into internal operands LW_{w'} = sum_w W_i[w,w'] L_w and
 * WR_{w'} = sum_{w''} W_{i+1}[w',w''] R_{w''}; the caller's buffers are not retained. */
int mrd_heff_set_env(mrd_heff* h, const double* lenv_dev, const double* renv_dev);
/* theta_out = H_eff theta_in (device pointers, complex128; must not overlap). prec:
 * MRD_PREC_FP64 runs FP64 grouped GEMMs, MRD_PREC_FF the same grouped GEMMs in float-float
 * arithmetic (~1e-13 relative); MRD_PREC_TF32 and MRD_PREC_BF16X3 run the same
 * contraction on the tcgen05 tensor cores with FP32 accumulation (complex products as four
 * real ones), operands repacked into 128-byte swizzled tiles: the folded environments once
 * after each mrd_heff_set_env, theta on every call; the result is returned in complex128. */
int mrd_heff_apply(mrd_heff* h, const double* theta_in_dev, double* theta_out_dev, int32_t prec);
/* Real flops of one H_eff application (8 per complex multiply-add), written to flops4:
 * [0] in the order of the definition (L step, W step, R step); [1] as executed by the
 * library, no padding counted; [2] and [3] the executed share of its step-1
 * (Z = LW theta) and step-2 (theta' = sum Z WR) grouped GEMMs. */
int mrd_heff_flops(const mrd_heff* h, double* flops4);
/* Kernel timing. With on != 0 every mrd_heff_apply records CUDA events around its two
 * grouped-GEMM launches on the context stream (no synchronisation). collect() waits for
 * the recorded work, returns the summed durations in ms of the step-1 and step-2 launches
 * and the number of applies recorded, and clears the record. */
int mrd_heff_timing(mrd_heff* h, int32_t on);
/* Execution options of an H_eff (value per option; returns MRD_E_ARG for an unknown option):
 *   MRD_OPT_GRAPH           1 (default): mrd_lanczos captures one Lanczos step (matvec,
 *                           reorthogonalisation, tridiagonal solve) as a CUDA graph and
 *                           replays it; 0: launches every kernel of every step.
 *   MRD_OPT_PER_TASK_LAUNCH 0 (default): each GEMM step of mrd_heff_apply is one grouped
 *                           persistent launch over all charge blocks; 1: one launch per task
 *                           (output block), the per-block baseline the grouped launch replaces.
 *   MRD_OPT_AUTOTUNE        1 (default): the first tensor-core application of a problem
 *                           class (precision, size of theta, number of tasks) times every
 *                           candidate tile configuration (columns per tile, pipeline stages,
 *                           task order) and keeps the fastest for the context; later H_effs
 *                           of the class reuse it; 0: the default configuration. */
/*   MRD_OPT_WAIT_LIMIT_US   1000000 (default): how long, in microseconds, a wait inside a
 *                           tensor-core GEMM (for a shared-memory stage, an accumulator or
 *                           the other warp roles) may last before the kernel gives up: it then
 *                           sets an error flag, waits for its own copies and MMAs in flight,
 *                           frees its tensor memory and returns. 0 gives up at the first wait,
 *                           before any copy or MMA is issued (a test of the error path).
 *                           Range 0 .. 60,000,000; MRD_E_ARG outside it. The flag is reported
 *                           as MRD_E_TIMEOUT by the next mrd_lanczos, mrd_heff_rayleigh or
 *                           mrd_heff_status, which clear it; the context stays usable. */
#define MRD_OPT_GRAPH 1
#define MRD_OPT_PER_TASK_LAUNCH 2
#define MRD_OPT_AUTOTUNE 3
#define MRD_OPT_WAIT_LIMIT_US 4
/*   MRD_OPT_REAL            0 (default); 1: the operands are real (MPO entries, which must then
 *                           be real, e.g. from MRD_BASIS_MIXED_REAL; environments; theta):
 *                           the tensor-core precisions drop the imaginary planes (TF32: one
 *                           MMA per K step instead of two, split BF16: two of half the width
 *                           instead of four) and write zero imaginary parts. The float-float and
 *                           FP64 paths are unchanged (their results are real for real inputs).
 *                           This is the real arithmetic the paper runs (Sec. IV.D, Eq. rot). */
#define MRD_OPT_REAL 5
int mrd_heff_set_option(mrd_heff* h, int32_t option, int64_t value);
/* Wait for the context stream and report a device-side wait of a tensor-core GEMM that gave
 * up since the last check: MRD_E_TIMEOUT (the flag is then cleared), else 0. */
int mrd_heff_status(mrd_heff* h);
/* Tensor-core tile configuration in use: cfg4 = {columns per tile, pipeline stages, task
 * order (0: charge order, 1: largest work first), source (0: default, 1: tuned on this
 * H_eff, 2: tuned earlier on the context)}; all -1 before the first tensor-core application. */
int mrd_heff_tc_config(const mrd_heff* h, int32_t* cfg4);
int mrd_heff_timing_collect(mrd_heff* h, double* ms_step1, double* ms_step2, int32_t* n_calls);

/* ------------------------------------------------------------------ eigensolver */

#define MRD_LANCZOS_MAX_ITER 60

/* Lowest eigenpair of H_eff by Lanczos with full reorthogonalisation (two classical
 * Gram-Schmidt passes per step), the standard DMRG eigensolver. theta_dev: start vector
 * on entry, normalised ground vector on exit (device, complex128, theta layout). Stops when
 * the lowest Ritz value changes by less than tol * |E|, when the Krylov space is exhausted,
 * or after max_iter (1..MRD_LANCZOS_MAX_ITER) matvecs. The matvecs use precision `prec`;
 * all vector arithmetic and the tridiagonal eigenproblem are FP64 on the device. Writes the
 * Ritz value to *energy and the number of matvecs to *iters. The workspace ((max+1)
 * vectors) is allocated on the first call and kept by the handle. */
int mrd_lanczos(mrd_heff* h, double* theta_dev, int32_t max_iter, double tol, int32_t prec, double* energy,
                int32_t* iters);
/* Rayleigh quotient E = <theta, H theta> / <theta, theta> with one matvec of precision
 * `prec` (FP64 on the device), and the relative residual |H theta - E theta| / |theta|. */
int mrd_heff_rayleigh(mrd_heff* h, const double* theta_dev, int32_t prec, double* energy, double* residual);

/* ------------------------------------------------------------------ two-site DMRG */

typedef struct {
  int32_t chi;               /* bond dimension: keep at most chi Schmidt values per bond     */
  double svd_cutoff;         /* drop Schmidt values below svd_cutoff * largest (e.g. 1e-14)  */
  int32_t lanczos_max_iter;  /* 1 .. MRD_LANCZOS_MAX_ITER                                    */
  double lanczos_tol;        /* relative change of the Ritz value that stops Lanczos         */
  int32_t prec;              /* MRD_PREC_* of the Lanczos matvecs                            */
  int32_t refine_iter;       /* > 0 with a reduced prec: FP64 Lanczos polish of the ground   */
                             /* vector, at most this many FP64 matvecs (iterative refinement) */
  double refine_tol;         /* relative Ritz-value change that stops the polish              */
  int32_t lanczos_restarts;  /* extra Lanczos runs restarted from the current ground vector   */
                             /* while the Ritz value still moves by more than lanczos_tol     */
  int32_t svd_mode;          /* MRD_SVD_*: arithmetic of the one-sided Jacobi sweeps          */
  int32_t refine_prec;       /* MRD_PREC_FP64 or MRD_PREC_FF: arithmetic of the refinement    */
                             /* matvecs, the environment updates and the GEMMs of the SVD     */
} mrd_dmrg_params;

/* Block SVD sweep arithmetic. The final sweeps stop when every column pair is orthogonal to
 * 1e-14 (FP64) or 5e-13 (float-float: pairs of FP32 numbers, ~48-bit products, on the FP32
 * pipes); FP32 pre-sweeps (to 1e-5, at most 8 sweeps) may precede them. */
#define MRD_SVD_F32_FF 0   /* FP32 pre-sweeps, float-float sweeps */
#define MRD_SVD_FF 1       /* float-float sweeps only             */
#define MRD_SVD_F32_F64 2  /* FP32 pre-sweeps, FP64 sweeps        */
#define MRD_SVD_F64 3      /* FP64 sweeps only                    */

/* Finite two-site DMRG state on the device for the MPO `mpo` (copied; it may be freed later) in the
 * charge sector (N = n_part, K = k_tot mod modulus). Starts from a seeded random MPS whose
 * entries are SplitMix64 draws (counter-based, seed `seed`): sites left of `center` are
 * left-canonical, the others right-canonical (orthonormalised by the block SVD), and the
 * left environments up to bond `center` and right environments from bond center+2 are
 * built. Bond sectors are the exactly reachable charges, each of dimension at most its exact
 * state count and chi (scaled down so every bond sums to at most chi); if caps/caps_off are
 * given, bond j only keeps the sectors listed in caps[3*caps_off[j] .. 3*caps_off[j+1]) as
 * (N, K, max dim) triplets (bonds with an empty list use the default). */
int mrd_dmrg_create(mrd_ctx* ctx, const mrd_mpo* mpo, int32_t n_part, int32_t k_tot, int32_t chi, uint64_t seed,
                    int32_t center, const int32_t* caps, const int64_t* caps_off, mrd_dmrg** out);
int mrd_dmrg_free(mrd_dmrg* d);
/* One two-site update at sites (i, i+1) (standard two-site DMRG): theta = M_i M_{i+1}, ground
 * state of H_eff by Lanczos, block SVD of theta by middle charge (the Schmidt decomposition,
 * Sec. III.C), truncation to chi with cutoff, renormalised Schmidt values; direction +1
 * moves the orthogonality centre right (A_i = U, M_{i+1} = S V^+, then L_{i+1}) and -1 left
 * (M_i = U S, B_{i+1} = V^+, then R_{i+1}). Needs L_i and R_{i+2}. With a reduced-precision
 * prec and refine_iter > 0 the Lanczos ground vector is polished by FP64 Lanczos started
 * from it (iterative refinement); the energy is then the FP64 Ritz value. Writes the energy
 * and the discarded weight. */
int mrd_two_site_update(mrd_dmrg* d, int32_t i, int32_t direction, const mrd_dmrg_params* p, double* energy,
                        double* trunc_err);
/* One sweep: two-site updates left to right over all bonds, then right to left (requires the
 * centre at site 0). Writes the last energy. */
int mrd_sweep(mrd_dmrg* d, const mrd_dmrg_params* p, double* energy);
/* Environment update of two-site DMRG (the paper relies on standard DMRG, its refs. W92,
 * S2005): with direction +1 the left environment of bond site+1 is rebuilt from that of bond
 * `site`, the MPS tensor A = site and the MPO site W:
 *   L'_{w'}[c', c] = sum_{w, a', a, s', s} conj(A[a', s', c']) L_w[a', a] W[w, w', s', s] A[a, s, c];
 * with direction -1 the right environment of bond `site` is rebuilt from that of bond site+1
 * and B = site:
 *   R'_w[c, c'] = sum_{w', b, b', s', s} B[c, s, b] R_{w'}[b, b'] conj(B[c', s', b']) W[w, w', s', s].
 * Block-sparse in the charges: only blocks with q_{c'} = q_c + c_{w'} (left) or
 * q_{c'} = q_c + c_w (right) exist, in the env layouts of this header. The tensor is used as it
 * is (an update leaves it left-canonical moving right and right-canonical moving left, which
 * makes the environment the projected Hamiltonian). The result replaces the state's
 * environment of that bond, readable with mrd_dmrg_env; two-site updates call the same code.
 * prec: MRD_PREC_FP64 (FP64 grouped GEMMs) or MRD_PREC_FF (float-float, ~1e-13 relative).
 * MRD_E_ARG for a site outside 0..n-2 (+1) or 1..n-1 (-1), MRD_E_STATE if the input
 * environment has not been built. */
int mrd_env_update(mrd_dmrg* d, int32_t site, int32_t direction, int32_t prec);
/* Options of a DMRG state:
 *   MRD_DMRG_OPT_ENV_FP32   0 (default): environments are stored in complex128; 1: stored in
 *                           complex64 (half the bytes, for the memory-bound scale of large
 *                           circumferences and bond dimensions). Setting it converts the
 *                           environments already built; later environment updates compute in
 *                           FP64 or float-float as before and round their result to complex64
 *                           for storage, and an update widens the two environments it reads
 *                           back to complex128 before folding them with the MPO. The rounding
 *                           (2^-24 relative per entry) enters the H_eff of later updates.
 * MRD_E_ARG for an unknown option. */
#define MRD_DMRG_OPT_ENV_FP32 1
/*   MRD_DMRG_OPT_REAL       1: real arithmetic (Sec. IV.D, Eq. rot): the MPO must be real (e.g.
 *                           MRD_BASIS_MIXED_REAL; MRD_E_ARG otherwise) and the option set before
 *                           the first update (MRD_E_STATE otherwise). The seeded random tensors
 *                           are replaced by their real parts and canonicalised again, the
 *                           environments rebuilt; every later H_eff is declared real
 *                           (MRD_OPT_REAL), and all tensors stay real. 0 switches it off. */
#define MRD_DMRG_OPT_REAL 2
/*   MRD_DMRG_OPT_SVD_PRESWEEPS  0 .. 64 (default 8): the largest number of FP32 Jacobi
 *                           pre-sweeps of the block SVD modes MRD_SVD_F32_* (they stop earlier
 *                           once no pair rotates); 0 leaves all work to the final sweeps.
 *                           Columns are set aside before the final sweeps (mrd_dmrg_svd_stats)
 *                           only after at least 8 pre-sweeps or converged ones. */
#define MRD_DMRG_OPT_SVD_PRESWEEPS 3
int mrd_dmrg_set_option(mrd_dmrg* d, int32_t option, int64_t value);
/* Device memory of a DMRG state: out4 = {bytes of the stored environments, environments
 * built, bytes of the MPS tensors, 1 if environments are stored in complex64}. */
int mrd_dmrg_memory(const mrd_dmrg* d, int64_t* out4);
/* Sectors of MPS bond `bond` (0..n) as (N, K, dim) triplets (sectors may be NULL). */
int mrd_dmrg_bond(const mrd_dmrg* d, int32_t bond, int32_t* n_sectors, int32_t* sectors);
/* Copy of MPS tensor `site` to the host (complex128). mode 0: blocks grouped by right
 * sector r, each a (rows (s, l) with l = r - q(s), s = 0 first) x d_r row-major matrix;
 * mode 1: grouped by left sector l, each a d_l x (columns (s, r), r = l + q(s)) matrix.
 * host may be NULL (only *mode and *len are set). */
int mrd_dmrg_site(mrd_dmrg* d, int32_t site, int32_t* mode, int64_t* len, double* host);
/* Copy of the left (side 0) or right (side 1) environment at `bond` in the layouts of this
 * header; *len = -1 if it is not built. */
int mrd_dmrg_env(mrd_dmrg* d, int32_t bond, int32_t side, int64_t* len, double* host);
/* Replace the data of MPS tensor `site` with host data in the layout mrd_dmrg_site reports
 * (same sectors and mode; *len complex128 values). The copy is enqueued on the context
 * stream (pinned host memory makes it asynchronous). */
int mrd_dmrg_set_site(mrd_dmrg* d, int32_t site, const double* host);
/* GEMM kernel timing of the updates: returns (and clears) the accumulated CUDA-event times in
 * ms of the tensor-core step-1 and step-2 launches and of the FP64 step-1 and step-2
 * launches, and the number of tensor-core and FP64 H_eff applications; then switches the
 * recording on (on != 0) or off. Arrays may be NULL. */
int mrd_dmrg_timing(mrd_dmrg* d, int32_t on, double* kernel_ms4, int64_t* applies2);
/* Wall time in ms of the phases of the last two-site update (each ends with a stream
 * synchronisation): [0] H_eff tables and environment fold, [1] theta, [2] Lanczos,
 * [3] block SVD and truncation, [4] new MPS tensors, [5] environment update; then [6] the
 * FP32 and [7] the FP64 Jacobi sweeps of its block SVD. */
int mrd_dmrg_phase_ms(const mrd_dmrg* d, double* ms8);
/* Block SVD of the last two-site update: out8 = {ms of the final (float-float or FP64) Jacobi
 * sweeps (CUDA events around them), column element-pairs whose overlap was tested (sum of the
 * column length over tested pairs), element-pairs rotated, final sweeps, ms of the FP32
 * pre-sweeps (0 without), svd_mode, columns that entered the final sweeps, columns of all
 * blocks}. With FP32 pre-sweeps and more columns than chi, columns whose norm after the
 * pre-sweeps is below half the chi-th largest column norm are set aside before the final
 * sweeps (their Schmidt weight is discarded by the truncation to chi in any case). */
int mrd_dmrg_svd_stats(const mrd_dmrg* d, double* out8);
/* Column pairs rotated in each Jacobi sweep of the last block SVD: n2[0] FP32 pre-sweeps, then
 * n2[1] final sweeps; the first cap counts (pre-sweeps first) are copied to out and, when ms
 * is not NULL, the host wall time of each sweep in ms (its launches up to the read-back of its
 * rotation count) to ms. */
int mrd_dmrg_svd_trace(const mrd_dmrg* d, int32_t cap, int32_t* out, double* ms, int32_t* n2);
/* Momentum-resolved entanglement spectrum (Sec. III.C): the Schmidt values lambda of the
 * bond cut by the last two-site update (*bond = i + 1 for an update of sites i, i+1), one per
 * kept Schmidt state, with the charges (N, K) of its left part in nk (2 per value). The values
 * of one sector are consecutive, sectors in increasing (N, K); sum lambda^2 = 1. They are the
 * norms of the centre tensor's rows (or columns, moving left) against the isometric canonical
 * factor; entanglement energies are -2 ln lambda. Call with nk = values = NULL for *n. */
int mrd_dmrg_schmidt(const mrd_dmrg* d, int32_t* bond, int64_t* n, int32_t* nk, double* values);
/* Energy, discarded weight and matvec count of the last two-site update; the count is the
 * reduced-precision (or FP64) Lanczos matvecs plus 1000 times the FP64 refinement matvecs. */
int mrd_dmrg_stats(const mrd_dmrg* d, double* energy, double* trunc_err, int32_t* lanczos_iters);

/* Issue rates measured on the context's device, for roofline fractions of the kernels that
 * run on the CUDA-core pipes (the float-float GEMM and Jacobi sweeps on FP32, the FP64 forms):
 * out4 = {FP32 fused multiply-add instructions per second, FP64 fused multiply-add
 * instructions per second, SM count, maximum SM clock in Hz}. Each rate is the best of 5
 * timed launches of independent multiply-add chains filling every SM; takes a few ms.
 * (The paper has no counterpart; this supports the measurements.) */
int mrd_measure_peaks(mrd_ctx* ctx, double* out4);

/* Capacity of the static scratch used by mrd_heff_apply_noalloc, in complex128 elements
 * (64 MiB). */
#define MRD_NOALLOC_Z_MAX_ELEMS (4194304)

/* theta_out = H_eff theta_in like mrd_heff_apply with MRD_PREC_FP64, but this call
 * allocates nothing: no cudaMalloc, cudaFree or other allocating routine. It is for callers
 * that may not allocate device memory when they need the product, for instance code whose
 * device memory is owned by an external pool that must see every allocation, or a thread
 * that must not touch the CUDA allocator while work is being captured elsewhere. (The paper
 * has no counterpart; this is an interface convenience.)
 *
 * The step-1 intermediate Z (normally a buffer allocated by mrd_heff_create) lives instead in
 * a static device array of MRD_NOALLOC_Z_MAX_ELEMS complex128 elements that every GPU which
 * loads this library keeps until the process exits. Problems whose Z is larger are rejected
 * with MRD_E_ARG and a message naming both sizes; use mrd_heff_apply for them. The first call
 * on a device looks up the array's device address (cudaGetSymbolAddress, with that device
 * current), so make that first call before any stream capture; the address is kept for the
 * life of the process and is not valid after a cudaDeviceReset (nor is any other handle). All calls share the one
 * array: two calls whose device work overlaps in time (different streams or contexts) race
 * and give wrong results; calls ordered on one stream are safe. theta_out is cleared by the
 * call; Z needs no clearing because step 2 reads only what step 1 of the same call wrote.
 * The handle must have its environments loaded (mrd_heff_set_env). */
int mrd_heff_apply_noalloc(mrd_heff* h, const double* theta_in_dev, double* theta_out_dev);

/* Table export for bit-exact checks. which = 0: middle sectors, 8 int64 per row
 * (N, K, rowdim, coldim, offset, row_off_s1=1, col_off_s2=1, flags); which = 1: left-env
 * blocks, 6 int64 (w, a, a', offset, rows, cols); which = 2: right-env blocks, 6 int64
 * (w, b, b', offset, rows, cols). If rows == NULL only *count is set. */
int mrd_heff_table(const mrd_heff* h, int32_t which, int64_t* rows, int64_t* count);

#ifdef __cplusplus
}
#endif
#endif /* MRDMRG_H */
