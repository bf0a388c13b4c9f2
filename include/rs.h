/*
 * rs.h -- C ABI of librs: range-separated (RS) tensor electrostatics for
 * rigid protein-ligand poses on one GB300 (sm_103a).
 *
 * Method: arXiv 2510.26611, "Fast tensor-based electrostatic energy
 * calculations in the perspective of protein-ligand docking problem".
 *   - rs_build_protein      : Algorithm TEP (Sec. 3.4): sinc sum of Gaussians for
 *                             1/r (Sec. 2, Eq. sinc), range split (Eq. Split_Tens),
 *                             shifted long-range Gaussians (Eq. Long-Range_Sum),
 *                             rank reduction by RHOSVD (TEP step 4, Sec. 4.1).
 *   - rs_energy_poses       : Algorithm PLIE (Sec. 3.4) over a batch of poses
 *                             (Lemma 3.3, Eq. EnergySum_ligand) plus the short-range
 *                             part (Def. 2.1) and the vdW constraint of
 *                             Eq. Energy_Min (Sec. 3.4).
 *   - rs_energy_grad_poses  : derivative of Eq. EnergySum_ligand with respect to the
 *                             rigid-body parameters (Sec. 3.3 forces; Sec. 4.2,
 *                             force on a rigid cluster, taken exactly).
 *
 * Conventions shared by every call
 *   - Units: Angstrom and elementary charge; energies in e^2/Angstrom.
 *   - The grid has n nodes per axis, x_i = -b + i*h, h = 2b/(n-1).
 *   - Ligand coordinates are re-centred on their unweighted geometric centre
 *     (Sec. 3.4); a pose's translation is the absolute position of that centre.
 *     Rotations act about the centre.  Quaternions are (w, x, y, z) and are
 *     normalised by the library; rotation vectors w give R = exp([w]x).
 *   - The caller owns every input and output buffer; the library owns handles
 *     (freed with the matching *_free / *_destroy).  Inputs are never modified.
 *   - mem_flags: RS_MEM_HOST (all array pointers are host memory; the call
 *     copies in, computes and copies out, and returns when results are in the
 *     output buffers) or RS_MEM_DEVICE (all array pointers are device memory on
 *     the context's GPU; the work is enqueued on `stream` and the call returns
 *     after enqueue).  `stream` is a cudaStream_t passed as void*, used exactly
 *     as given: NULL is the CUDA default stream.  Work of one call is ordered
 *     after earlier work on that stream.
 *   - Errors: every call returns an rs_status; on failure nothing is written to
 *     the outputs that is meant to be used and rs_last_error() gives a message
 *     (thread-local).  No exception crosses the ABI.  No call aborts.
 */
#ifndef RS_H_
#define RS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int rs_status;
#define RS_OK               0
#define RS_ERR_INVALID     -1   /* bad argument: null pointer, size out of range */
#define RS_ERR_OOM         -2   /* device or host allocation failed / budget exceeded */
#define RS_ERR_CUDA        -3   /* a CUDA runtime call failed */
#define RS_ERR_TIMEOUT     -4   /* a bounded wait ran out */
#define RS_ERR_BUSY        -5   /* resource temporarily unavailable (queue full) */
#define RS_ERR_NOT_READY   -6   /* result not available yet (serving poll) */
#define RS_ERR_UNSUPPORTED -7   /* size or option outside what this build handles */

#define RS_MEM_HOST   0
#define RS_MEM_DEVICE 1

/* Bits of the per-pose flag byte. */
#define RS_FLAG_CLASH        1  /* some ligand-protein distance < sigma (Eq. Energy_Min) */
#define RS_FLAG_OUT_OF_GRID  2  /* some ligand atom outside [-b, b]^3: clamped to the edge cell */

typedef struct rs_ctx rs_ctx;
typedef struct rs_protein rs_protein;

/* Parameters of Algorithm TEP (Sec. 3.4: grid size n, box, vdW distance sigma)
 * and of the sinc quadrature and reduction the paper leaves open.  Fill with
 * rs_params_default() and override. */
typedef struct rs_params {
    int32_t n;          /* grid nodes per axis, 3 <= n <= 16385                       */
    double  b;          /* box half-width: the grid spans [-b, b]^3, b > 0            */
    double  sigma;      /* van der Waals distance (Remark 3.1), > 0                   */
    int32_t R_l;        /* number of long-range sinc terms, 2 <= R_l <= 64            */
    double  r_min;      /* smallest distance the quadrature targets (default 0.5)     */
    double  tau;        /* narrowest long-range Gaussian has t*sigma = tau (default 4)*/
    double  short_tol;  /* short-range cutoff: r*sum_short a_k e^{-t_k^2 r^2} <= tol  */
    int32_t tucker_cap; /* 0: keep the unreduced canonical rank N*R_l; >0: RHOSVD to
                           Tucker ranks <= tucker_cap (<= 32)                          */
    double  eps_r;      /* RHOSVD keeps singular values > eps_r * s_1 (default 1e-7)  */
    int32_t galerkin;   /* 0: collocation (factor entries are the Gaussians' values at
                           the nodes); 1: Galerkin (their averages over the node's cell
                           [x_i - h/2, x_i + h/2], Sec. 2, Eq. galten), canonical form
                           only (tucker_cap = 0, else RS_ERR_UNSUPPORTED)               */
} rs_params;

/* Read-only description of a built protein potential. */
typedef struct rs_protein_info {
    int32_t n, N, R_l, K;       /* grid, atoms, long-range terms, total sinc terms  */
    double  b, h, sigma, r_c;   /* box, spacing, vdW distance, short-range cutoff   */
    double  h_s, quad_err;      /* quadrature step and measured max rel. error of 1/r */
    int32_t kind;               /* 0 = canonical (unreduced), 1 = Tucker            */
    int32_t rank[3];            /* canonical: {R, R, R}; Tucker: r_1, r_2, r_3       */
    double  sv_gap[3];          /* Tucker: s_r / s_{r+1} per axis (0 if r = n)      */
    double  sv_tail[3];         /* Tucker: (sum_{i>r} s_i^2)^(1/2) / s_1 per axis    */
    size_t  device_bytes;       /* device memory held by the handle                 */
} rs_protein_info;

/* ---------------------------------------------------------------- context */
void        rs_params_default(rs_params* p);
/* Creates a context on CUDA device `device` (made current for every call that
 * uses the context).  *out receives the handle.  A context owns device scratch
 * (prepared ligand, staging, the per-atom arrays of the pose path) that every
 * call through it reuses: calls through one context must not run on the GPU at
 * the same time (issue them on one stream, or order the streams); use one
 * context per concurrent stream.  Growing the scratch frees the old buffer,
 * which waits for the device. */
rs_status   rs_ctx_create(int device, rs_ctx** out);
void        rs_ctx_destroy(rs_ctx* ctx);
/* Message of the last failing call on this thread ("" if none). */
const char* rs_last_error(void);
/* Library version string. */
const char* rs_version(void);

/* ------------------------------------------------------- Algorithm TEP */
/* Builds the RS potential of a protein (Algorithm TEP, Sec. 3.4).
 *   N     : number of protein atoms, 1 <= N <= 2^22
 *   xyz   : [N][3] float64 positions (Angstrom); q: [N] float64 charges (e)
 *   params: see rs_params
 *   mem_flags/stream: where xyz and q live; the build runs on `stream` (after
 *           earlier work on it) and the call returns when the handle is ready.
 * On success *out owns the device-resident factors, the sinc table and a
 * cell list of the atoms; free it with rs_protein_free. */
rs_status rs_build_protein(rs_ctx* ctx, int32_t N, const double* xyz, const double* q,
                           const rs_params* params, int mem_flags, void* stream,
                           rs_protein** out);
void      rs_protein_free(rs_protein* p);
rs_status rs_protein_get_info(const rs_protein* p, rs_protein_info* out);
/* Copies the sinc table: t[K], a[K] (float64) and is_long[K] (uint8), K from info. */
rs_status rs_protein_get_table(const rs_protein* p, double* t, double* a, uint8_t* is_long);

/* ------------------------------------------------------ Algorithm PLIE */
/* Energies of P rigid poses of one ligand (Algorithm PLIE; Lemma 3.3):
 *   E[p] = sum_j q_j (phi_long + phi_short)(R_p y_j + t_p)
 * phi_long is the long-range RS tensor interpolated trilinearly (per 1D factor)
 * at the atom, phi_short the short-range Gaussians of protein atoms closer than
 * r_c, y_j the ligand atoms about their centre.
 *   L        : ligand atoms, 1 <= L <= 4096; lig_xyz [L][3], lig_q [L] float64
 *   P        : poses, 0 <= P <= 2^31-1 (P = 0 is a no-op)
 *   quat     : [P][4] float64 (w,x,y,z); trans: [P][3] float64
 *   E_out    : [P] float64;  flags_out: [P] uint8 (RS_FLAG_* bits), may be NULL
 * The long range is evaluated on the FP32 pipes in float-pair arithmetic
 * (about 48 significant bits); atom positions, the short range and the vdW
 * decisions near sigma are FP64; pose sums are FP64.  For a Tucker-reduced
 * protein the ligand atoms of all poses are grouped by grid cell first (device
 * scratch of about 110 bytes per pose-atom, 190 with gradients, in chunks of at
 * most 2^23 pose-atoms); the results do not depend on that grouping. */
rs_status rs_energy_poses(rs_ctx* ctx, const rs_protein* prot, int32_t L,
                          const double* lig_xyz, const double* lig_q, int64_t P,
                          const double* quat, const double* trans,
                          double* E_out, uint8_t* flags_out, int mem_flags, void* stream);

/* Energies and exact gradients for poses given by rotation vectors:
 *   dE/dt = sum_j q_j grad phi(x_j)
 *   dE/dw = J_l(w)^T sum_j q_j (R y_j) x grad phi(x_j)   (J_l: SO(3) left Jacobian)
 * grad phi is the derivative of the piecewise-trilinear interpolant (difference
 * quotient of adjacent factor rows, Eq. Gradients_Tens) plus the analytic
 * derivative of the short-range Gaussians; it is 0 along an axis on which the
 * atom is outside the grid.
 *   rotvec: [P][3]; trans: [P][3]; dE_dt, dE_dw: [P][3] float64 outputs. */
rs_status rs_energy_grad_poses(rs_ctx* ctx, const rs_protein* prot, int32_t L,
                               const double* lig_xyz, const double* lig_q, int64_t P,
                               const double* rotvec, const double* trans,
                               double* E_out, double* dE_dt, double* dE_dw,
                               uint8_t* flags_out, int mem_flags, void* stream);

/* A molecular complex against a ligand molecule (Sec. 5.1, Eq. EnergySum_Mcomplex):
 * E_p = sum_j q_j (phi_1 + ... + phi_nmol)(x_j), each phi_i the RS potential of
 * molecule mols[i] (each on its own grid and parameters, Tucker or canonical); a pose's
 * flags are the OR of its flags against every molecule.  Arguments as for
 * rs_energy_poses; 1 <= nmol <= 64.  Energies equal the sum, in molecule order, of
 * rs_energy_poses over the molecules. */
rs_status rs_energy_poses_complex(rs_ctx* ctx, int32_t nmol, const rs_protein* const* mols, int32_t L,
                                  const double* lig_xyz, const double* lig_q, int64_t P,
                                  const double* quat, const double* trans, double* E_out,
                                  uint8_t* flags_out, int mem_flags, void* stream);

/* Local-box handle: scheme (C) of Sec. 3.2 (Table 1).  The Tucker potential of
 * `parent` restricted to the grid nodes of the box [lo, hi] (Angstrom, per axis; the
 * interpolation cells that meet the box, at most 511 per axis) and re-truncated by an
 * HOSVD of that node tensor: per axis rank r = #{s_i > eps s_1} (r_1, r_2 <= 32).
 * Node-tensor error <= s_1 sqrt(sum over axes of sv_tail^2) (rs_protein_get_info
 * reports ranks, sv_tail and sv_gap of the local HOSVD).  The handle evaluates like
 * any Tucker protein on the same grid; an atom outside the box's cells is flagged
 * out of grid (bit 1) and its value is meaningless.  It shares the parent's
 * short-range data: rs_protein_free on the parent is deferred until its local
 * handles are freed (handles of one family must not be freed concurrently).
 * RS_ERR_INVALID for a canonical or local parent, an empty box or eps not in [0, 1).
 * A local-box handle is evaluated by rs_energy_poses, rs_energy_grad_poses, rs_pgd_run,
 * rs_fd_forces_poses, rs_ppiem_scan and rs_energy_poses_complex (the box flags are
 * set by a pass after the pose kernels); rs_batch_create and rs_energy_poses_noalloc
 * return RS_ERR_UNSUPPORTED for it. */
rs_status rs_protein_local_box(rs_ctx* ctx, rs_protein* parent, const double* lo, const double* hi,
                               double eps, rs_protein** out);

/* Add-and-compress: the long-range Tucker tensors of several molecules on one grid,
 * summed and re-truncated into one Tucker handle (Algorithm TEP, step 4, Sec. 3.4:
 * sums of Tucker tensors re-compressed by an HOSVD of the small core; Sec. 5.1, the
 * complex potential of Eq. EnergySum_Mcomplex as one tensor).  With T_p = beta_p x_l
 * V_l^(p) the parts' tensors, per axis [V_l^(1) ... V_l^(count)] = Q_l R_l (thin QR,
 * FP64 on the host; a column within 1e-12 of the span of the previous ones gets a
 * zero Q column), C = sum_p beta_p x_l R_l[:, columns of p], and the HOSVD of C
 * keeps per axis r_l = #{s_i > eps_r s_1} (1 <= r_l <= tucker_cap) leading singular
 * vectors U_l: V_l = Q_l U_l, core = C x_l U_l^T, then the cardinal basis and
 * evaluation tables as rs_build_protein makes them.  Long-range error (Frobenius, on
 * the grid) <= s_1 sqrt(sum over axes of sv_tail^2) (rs_protein_get_info: ranks,
 * sv_tail and sv_gap of this HOSVD).  The short range is that of
 * the union of the parts' atoms.
 *   parts: count (1..16) Tucker-reduced handles (not local-box handles) built on
 *   this context's device with the same n, b, sigma, R_l and sinc table; the sum of
 *   their ranks per axis <= 128 and of their atoms <= 2^22.  The parts are only read
 *   and stay owned by the caller; *out is a new handle (free with rs_protein_free).
 *   stream: the CUDA stream of the device work (NULL: the default stream); the call
 *   synchronises it before returning.
 * RS_ERR_INVALID for a NULL or mismatched part, count, tucker_cap not in [1, 32]
 * or eps_r not in [0, 1); RS_ERR_OOM / RS_ERR_CUDA as for
 * rs_build_protein (no handle is returned then). */
rs_status rs_protein_add_compress(rs_ctx* ctx, const rs_protein* const* parts, int32_t count, int32_t tucker_cap,
                                  double eps_r, void* stream, rs_protein** out);

/* The paper's finite-difference force and its rigid-cluster resultants, for
 * comparison with the exact gradient of rs_energy_grad_poses.
 *   Per atom l and axis i (Eq. differ_ligand, Sec. 3.3):
 *     F_{l,i} = q_l (phi(x_l) - phi(x_l - h e_i)) / h,
 *   phi the RS potential (long + short range), h the grid step when h = 0.  The
 *   quotient is taken as printed, so F_l approximates +grad of the energy.
 *   With r_l = R y_l (offset from the ligand centre x0 = the translation) and
 *   v_l = r_l / |r_l|, the pose outputs are
 *     E_out    [P]    sum_l q_l phi(x_l)
 *     F_out    [P][3] sum_l F_l                          (compare with dE/dt)
 *     F0_out   [P][3] sum_l (F_l . v_l) v_l              (Eq. Field_Xcenter, Sec. 5.2)
 *     Fphi_out [P][3] sum_l (|r_l| / r0) (F_l - (F_l . v_l) v_l)   (Eq. Field_phi)
 *     M_out    [P][3] sum_l r_l x F_l   (J_l(w)^T M compares with dE/dw)
 *   An atom at the centre (r_l = 0) puts all of F_l into F0.  r0 = 0 takes the RMS
 *   distance of the ligand atoms from their centre (Fphi = 0 if that is 0 too).
 * Each pose costs four evaluations of the potential at every atom (the pose and
 * its translations by -h e_i), on the cell-grouped path: the protein must be
 * Tucker-reduced (RS_ERR_UNSUPPORTED otherwise).  rotvec, trans: [P][3]; h, r0 >= 0
 * and finite (RS_ERR_INVALID otherwise); flags_out may be NULL; mem_flags and
 * stream as for rs_energy_poses. */
rs_status rs_fd_forces_poses(rs_ctx* ctx, const rs_protein* prot, int32_t L,
                             const double* lig_xyz, const double* lig_q, int64_t P,
                             const double* rotvec, const double* trans, double h, double r0,
                             double* E_out, double* F_out, double* F0_out, double* Fphi_out,
                             double* M_out, uint8_t* flags_out, int mem_flags, void* stream);

/* Pose scan of Algorithm PPIEM (Sec. 3.4, steps A0-A7).
 *   Orbit directions (A0, A5): u_d at polar angle (a + 1/2) pi / n_theta and azimuth
 *   2 pi b / n_phi, d = a n_phi + b (D = n_theta n_phi <= 65535).  Self-rotations (A4):
 *   the caller's unit quaternions quats [n_rot][4] (w, x, y, z).  x_P [3]: the centre
 *   the ligand approaches (A2); NULL takes the protein's geometric centre.
 *   Contact (A3): for each (d, r) the ligand centre moves along x_P + s u_d from far
 *   outside; s*_dr is the first s at which a ligand-protein distance reaches sigma,
 *   the largest c + sqrt(sigma^2 - q) over atom pairs with q < sigma^2, where
 *   w = x_m - x_P - R_r y_j, c = u_d . w, q = |w|^2 - c^2 (FP64; -inf if no pair
 *   blocks).  The pose (q_r, x_P + (s*_dr + margin sigma) u_d) (margin 0: 1e-6) is
 *   evaluated as by rs_energy_poses.
 *   Outputs: s_out, E_out, flags_out [D][n_rot] (each may be NULL; no contact:
 *   s = -inf, E = +inf, flag 4); E_best [D] lowest feasible energy of direction d
 *   (+inf if none), rot_best [D] its rotation (lowest index among ties, -1 if none),
 *   t_best [D][3] its translation; is_min [D] 1 where E_best[d] is a local minimum
 *   over the neighbours a +- 1 (no wrap) and b +- 1 (wrapping), ties to the lower d.
 * Device scratch ~16 D N + 100 D n_rot bytes plus the pose path's.  mem_flags and
 * stream as for rs_energy_poses. */
rs_status rs_ppiem_scan(rs_ctx* ctx, const rs_protein* prot, int32_t L, const double* lig_xyz,
                        const double* lig_q, int32_t n_theta, int32_t n_phi, int32_t n_rot,
                        const double* quats, const double* x_P, double margin, double* s_out,
                        double* E_out, uint8_t* flags_out, double* E_best, int32_t* rot_best,
                        double* t_best, uint8_t* is_min, int mem_flags, void* stream);

/* Constrained energy minimisation of Eq. Energy_Min (Sec. 3.4) by projected
 * gradient descent on (translation, rotation vector), `nsteps` steps for every
 * pose.  Each step: gradient g by rs_energy_grad_poses; trial poses
 * (t - s eta_t g_t/|g_t|, w - s eta_r g_w/|g_w|) with s = 1, 1/2, ..., 2^-max_halvings;
 * the first trial that is feasible (no flag) and does not raise E replaces the
 * pose, otherwise the pose is kept.  All arrays are device memory:
 *   rotvec, trans : [P][3] in/out (updated in place)
 *   E_out, flags_out : [P] energy and flags of the final poses
 *   accepted_out  : [P] int32, halving level accepted at the last step, -1 if kept
 * Runs on the context's stream, ordered after `stream` and before later work on
 * it; returns when the work is enqueued. */
rs_status rs_pgd_run(rs_ctx* ctx, const rs_protein* prot, int32_t L, const double* lig_xyz,
                     const double* lig_q, int64_t P, double* rotvec, double* trans,
                     int32_t nsteps, double eta_t, double eta_r, int32_t max_halvings,
                     double* E_out, uint8_t* flags_out, int32_t* accepted_out, void* stream);

/* ------------------------------------------------------------- batching */
/* One protein-ligand pair of a batch.  All arrays are device memory on the
 * context's GPU; the pair's protein must be Tucker-reduced (tucker_cap > 0). */
typedef struct rs_pair {
    const rs_protein* prot;
    int32_t L;              /* ligand atoms, 1..4096                              */
    const double* lig_xyz;  /* [L][3], read once by rs_batch_create              */
    const double* lig_q;    /* [L]                                               */
    int64_t P;              /* poses                                             */
    const double* quat;     /* [P][4] (w,x,y,z), read at every rs_batch_run      */
    const double* trans;    /* [P][3], read at every rs_batch_run                */
    double* E_out;          /* [P]                                               */
    uint8_t* flags_out;     /* [P] or NULL                                       */
} rs_pair;

typedef struct rs_batch rs_batch;

typedef struct rs_batch_info {
    int32_t npairs, ngroups;  /* pairs; groups (one per padded Tucker rank)       */
    int32_t nitems;           /* per-block path: work items over its groups       */
    int32_t grid;             /* per-block path: persistent CTAs over its groups  */
    int32_t threads;          /* per-block path: threads per CTA (first group)    */
    int32_t atoms_per_item;   /* per-block path: target atoms per item           */
    double  tune_ms;          /* device time the autotuner spent                  */
    int32_t mode;             /* first group: 0 per-block, 1 cell-grouped, 2 pair
                                 by pair through the single-pair cell-grouped path,
                                 3 the same with pairs on concurrent streams       */
    int32_t warps_per_cta;    /* cell-grouped: warps per CTA of the W-form kernel */
    int64_t chunk_atoms;      /* cell-grouped: pose-atoms per chunk (at most)     */
    int32_t nchunks;          /* cell-grouped: chunks over its groups             */
    int32_t streams;          /* first group: concurrent streams (mode 3), else 1 */
} rs_batch_info;

/* Algorithm PLIE (Sec. 3.4) for many pairs of uneven size, grouped by padded
 * rank and captured once in a CUDA graph.  Per group either the cell-grouped
 * multi-pair pipeline (pose-atoms of all pairs sorted by (pair, grid cell)) or one
 * persistent per-block launch runs.  autotune = 1: the path and its shape (chunk
 * size, or threads per CTA and atoms per work item) are chosen by timing the
 * candidates (the per-block shapes, the cell-grouped pipeline, the pairs one by
 * one through the single-pair cell-grouped path, and that path with the pairs spread
 * over 2 or 4 concurrent streams, longest first onto the least-loaded stream, as
 * parallel branches of the graph) on all of the group's poses (this writes the output
 * arrays; cached per padded rank for the process); 0: the cell-grouped pipeline;
 * 2: the per-block launch with its default shape; 3: pair by pair through the
 * single-pair path; 4: that path on 4 concurrent streams (scratch per stream).
 * Ligands are prepared now;
 * poses are read from the given pointers at each rs_batch_run, so a caller may
 * rewrite them in place between runs.  Device scratch: about 110 bytes per
 * pose-atom of the largest chunk (at most 2^23 pose-atoms), once per stream in
 * mode 3.  Flags equal rs_energy_poses'; energies equal them bit for bit in modes 2
 * and 3 (each pair through the plain call's own dispatch) and where the other paths
 * take the same W form (tensor-core or float-pair, chosen per launch from its atoms
 * per cell), and within ~2e-8 relative otherwise. */
rs_status rs_batch_create(rs_ctx* ctx, int32_t npairs, const rs_pair* pairs, int32_t autotune,
                          rs_batch** out);
/* Replays the batch's graph on `stream` (NULL = the CUDA default stream). */
rs_status rs_batch_run(rs_batch* batch, void* stream);
void      rs_batch_free(rs_batch* batch);
rs_status rs_batch_get_info(const rs_batch* batch, rs_batch_info* out);

/* Same energies and flags as rs_energy_poses, for callers that must not cause any
 * device allocation during the call (for example a thread that may never run
 * cudaMalloc/cudaFree because those can synchronise the device, or a plug-in whose
 * host application owns all device memory).  The paper has no counterpart: this
 * is an interface choice.  Differences from rs_energy_poses:
 *   - every array pointer is device memory on the protein's GPU, or managed
 *     memory (no host mode); anything else (a host pointer, another GPU's memory)
 *     returns RS_ERR_INVALID before any launch; no context is needed; the call sets the protein's device current and
 *     enqueues on `stream` (NULL = the CUDA default stream);
 *   - the per-call scratch is a fixed array in the library's device image
 *     (288 KiB on every GPU that loads the library, kept until exit), so
 *     L may be at most 4096; larger L returns RS_ERR_UNSUPPORTED;
 *   - the first call on a device looks the array's address up once; make that
 *     first call before any stream capture;
 *   - all calls share the array and it keeps the last call's contents (each call
 *     writes everything it reads first), so calls that overlap on the GPU, e.g.
 *     on two streams at once, race and must be serialised by the caller;
 *   - no timing events are recorded for these launches (the launch counter
 *     still counts them). */
rs_status rs_energy_poses_noalloc(const rs_protein* prot, int32_t L, const double* lig_xyz,
                                  const double* lig_q, int64_t P, const double* quat,
                                  const double* trans, double* E_out, uint8_t* flags_out,
                                  void* stream);

/* -------------------------------------------------------------- serving */
/* A request loop with continuous batching (the paper has no counterpart: this is
 * the deployment of Algorithm PLIE for a stream of docking jobs).  A server owns
 * its own context on one GPU and one scheduler thread.  Requests of any protein,
 * ligand and grid size are queued by rs_serve_submit; the scheduler admits them in
 * arrival order while a device-memory budget allows, keeps each protein's RS factors
 * resident (keyed by protein_id; least recently used idle proteins are evicted
 * under memory pressure), and launches all newly admitted requests together as one
 * batched pose launch (one per padded Tucker rank), on alternating streams, so
 * requests that arrive while others run on the GPU are admitted and overlap with
 * them.  A request's energies and flags equal rs_energy_poses bit for bit, alone or
 * in any mix. */
typedef struct rs_server rs_server;

typedef struct rs_request {
    uint64_t protein_id;     /* cache key; 0: build for this request only       */
    int32_t N;               /* protein atoms (read only when the key misses)   */
    const double* prot_xyz;  /* [N][3] host                                     */
    const double* prot_q;    /* [N] host                                        */
    rs_params params;        /* Algorithm TEP parameters of the protein         */
    int32_t L;               /* ligand atoms, 1..4096                           */
    const double* lig_xyz;   /* [L][3] host                                     */
    const double* lig_q;     /* [L] host                                        */
    int64_t P;               /* poses, 0..2^26                                  */
    const double* quat;      /* [P][4] host (w,x,y,z)                           */
    const double* trans;     /* [P][3] host                                     */
} rs_request;

typedef struct rs_result {
    rs_status status;        /* RS_OK, RS_ERR_OOM (over budget / allocation failed), ... */
    int64_t t_submit_ns;     /* steady-clock times: submitted, admitted,        */
    int64_t t_admit_ns;      /* its launch enqueued, results copied out         */
    int64_t t_start_ns;
    int64_t t_end_ns;
    char message[160];       /* error text when status != RS_OK                 */
} rs_result;

typedef struct rs_serve_params {
    uint64_t mem_budget_bytes;     /* device bytes for factors + request buffers; 0: half
                                      of the free device memory at creation             */
    int32_t max_queue;             /* queued requests before submit returns RS_ERR_BUSY  */
    int32_t max_inflight_launches; /* launches on the GPU at once (>= 1)                 */
    int32_t idle_wait_ms;          /* scheduler sleep when idle                          */
    int32_t inject_alloc_failures; /* test hook: fail the next k device allocations      */
    int64_t group_min_atoms;       /* a Tucker request joins the cell-grouped pipeline when
                                      it has at least this many pose-atoms and ...       */
    double  group_atoms_per_cell;  /* ... at least this many per axis-3 grid cell; other
                                      requests take the per-block kernel (both >= 0)     */
    int32_t hold_builds;           /* test hook: nonzero keeps protein builds from
                                      starting until rs_serve_release_builds            */
} rs_serve_params;

typedef struct rs_serve_stats {
    uint64_t done, failed;         /* finished requests                              */
    uint64_t launches;             /* batched launches                               */
    uint64_t builds, cache_hits;   /* protein builds; requests served from the cache */
    uint64_t evictions;            /* cached proteins freed under memory pressure    */
    uint64_t queued, cached_proteins;
    uint64_t budget_bytes, used_bytes;
    double   mean_requests_per_launch;
} rs_serve_stats;

void      rs_serve_params_default(rs_serve_params* p);
/* Checks a request's sizes and pointers without a GPU (RS_OK or RS_ERR_INVALID). */
rs_status rs_request_validate(const rs_request* r);
rs_status rs_serve_create(int device, const rs_serve_params* params, rs_server** out);
/* Queues a request.  Every pointer of the request and E_out [P] / flags_out [P]
 * (may be NULL) are host memory owned by the caller, which keeps them valid and
 * untouched until the request is finished (poll/wait returns it) or cancelled.
 * Returns RS_ERR_BUSY when the queue is full. */
rs_status rs_serve_submit(rs_server* s, const rs_request* r, double* E_out, uint8_t* flags_out,
                          uint64_t* req_id);
/* RS_ERR_NOT_READY while pending; otherwise RS_OK and fills `out` (may be NULL)
 * and releases the request id.  The request's own outcome is out->status. */
rs_status rs_serve_poll(rs_server* s, uint64_t req_id, rs_result* out);
/* Like poll, waiting at most timeout_ms (RS_ERR_TIMEOUT if still pending). */
rs_status rs_serve_wait(rs_server* s, uint64_t req_id, int32_t timeout_ms, rs_result* out);
/* Removes a request that has not been admitted yet (RS_ERR_BUSY once admitted). */
rs_status rs_serve_cancel(rs_server* s, uint64_t req_id);
/* Lets protein builds start on a server created with hold_builds (a test hook:
 * requests of proteins that are not resident stay queued until then). */
rs_status rs_serve_release_builds(rs_server* s);
rs_status rs_serve_get_stats(rs_server* s, rs_serve_stats* out);
/* Finishes launched work, drops queued requests and frees everything. */
void      rs_serve_destroy(rs_server* s);

/* ----------------------------------------------------------- diagnostics */
/* The host FP64 symmetric eigensolver the Tucker build uses for its Rayleigh-Ritz
 * step (Householder tridiagonalisation + implicit QL), exported so that it can be
 * tested without a GPU.  A: n x n row-major (its symmetric part is used), host
 * memory; lam: [n] eigenvalues in descending order; W: n x n row-major, column c
 * the unit eigenvector of lam[c].  RS_ERR_UNSUPPORTED if the iteration does not
 * converge. */
rs_status rs_symeig_host(int32_t n, const double* A, double* lam, double* W);
/* The host FP64 thin QR rs_protein_add_compress uses for the stacked factor matrices
 * (Algorithm TEP step 4), exported so that it can be tested without a GPU: classical
 * Gram-Schmidt, a column projected out again while a pass removes more than half of
 * what is left (at most three passes), and a column left with at most 1e-12 of its
 * norm taken as dependent (zero column of Q, R[j][j] = 0).  A: n x k, column-major
 * (column j at A + j n), host memory, overwritten by Q; R: k x k row-major, upper
 * triangular, written; A = Q R to rounding.  RS_ERR_INVALID for n < 1, k not in
 * [1, 4096] or a NULL pointer. */
rs_status rs_qr_host(int32_t n, int32_t k, double* A, double* R);
/* These have no counterpart in the paper: they support measurement.
 * Number of kernels this library has launched in the process (all devices). */
unsigned long long rs_stats_kernel_launches(void);
/* Per-kernel device timing: mode 0 off, 1 the pose kernels and the heavy build
 * kernels, 2 every kernel.  While on, each timed launch is bracketed by a CUDA
 * event pair recorded on the stream the kernel runs on (a small overhead). */
rs_status rs_timing_enable(int mode);
/* Drops all recorded timings (waits for pending events first). */
rs_status rs_timing_reset(void);
/* Number of kernel names with recorded timings. */
int       rs_timing_count(void);
/* Timing record `index` (0 <= index < rs_timing_count()): kernel name (copied,
 * NUL-terminated, at most name_len bytes), total device milliseconds, launch
 * count, and the summed algorithmic work the launches reported (FLOPs or bytes,
 * per kernel; see the library's design notes).  Waits for pending events. */
rs_status rs_timing_get(int index, char* name, size_t name_len, double* total_ms,
                        unsigned long long* launches, double* work);

/* Long-range (W form, Sec. 3 Tucker interpolation) kernel of the cell-grouped pose
 * paths that rs_energy_poses, rs_energy_grad_poses, rs_batch_run and the server
 * take for large calls: mode 1 (default) runs the per-cell contraction on the
 * tensor cores (tcgen05 MMAs on exact BF16 slices, ~2^-33 relative accuracy of each
 * contraction) for launches whose axis-3 grid cells hold at least 96 pose-atoms on
 * average, and in float-pair arithmetic on the FP32 pipes (~2^-47) below that;
 * mode 0 always runs the float-pair kernel.  Both agree with the FP64 definition far inside the 1e-5 energy
 * tolerance; the per-block path of small calls is float-pair in both modes.
 * Process-wide; takes effect for launches (and batch plans) made afterwards.
 * Returns the previous mode. */
int       rs_set_wform_kernel(int mode);
/* GEMM-shaped steps of the Tucker build (RHOSVD, Sec. 1, Algorithm TEP step 4): the
 * block products Y = G Q of the subspace iteration and the projections of the
 * shifted Gaussians on the factor basis.  Mode 1 (default) runs them on the tensor
 * cores (tcgen05 MMAs on six exact BF16 slices per operand, exact FP32 sums per K
 * chunk, ~2^-45 of the chunk's row and column maxima; G Q for grids up to 4097 and
 * block sizes that are multiples of 16); mode 0 runs the float-pair kernels on the
 * FP32 pipes (~2^-47).
 * Process-wide; takes effect for builds started afterwards.  Returns the previous
 * mode. */
int       rs_set_build_gemm_kernel(int mode);
/* Number of tensor-core tiles on `device` whose MMAs did not complete within the
 * kernel's bounded wait (their energies were set to NaN); 0 in normal operation. */
rs_status rs_tc_error_count(int device, int32_t* out);
/* Work counters of the cell-grouped atoms kernel (short range, Def. 2.1 with the
 * vdW check of Eq. Energy_Min) on `device` since the last reset, for energy
 * (grad = 0) or gradient (grad = 1) launches: counts[0] pose-atoms evaluated,
 * counts[1] protein-atom candidates screened, counts[2] near pairs evaluated in
 * pair arithmetic; *fp32_ops the algorithmic FP32 pipe operations these amount to
 * (the library's work model of that kernel).  Synchronises the device; reset != 0
 * zeroes the counters. */
rs_status rs_diag_short_counts(int device, int grad, uint64_t* counts, double* fp32_ops, int reset);
/* Diagnostics of the float-pair exponential of the build's Gaussian sums (Sec. 2,
 * the shifted Gaussians of the factor assembly): out[i] = exp(x[i]) evaluated on the
 * GPU from the pair nearest x[i] (|x[i]| <= 80; ~2^-46 relative for x[i] >= -60, where
 * both words of the result are normal floats), returned as FP64.  Synchronous. */
rs_status rs_diag_pair_exp(int32_t n, const double* x, double* out);
/* Launch shape of the latest tensor-core W-form launch in the process: CTAs,
 * dynamic shared memory per CTA (bytes) and CTAs per SM the occupancy allows. */
rs_status rs_diag_tc_launch(int64_t* grid, int64_t* smem, int32_t* per_sm);
/* Diagnostics of the tensor-core contraction alone: for one cell with W, D
 * (RP x RP, row-major FP64, host) and `rows` <= 128 rows v (rows x RP, host), computes
 * X = v W^T and Xd = v D^T (rows x RP, host) by the same slicing, MMAs and
 * combination the pose kernels use.  RP in {4, 8, ..., 32}.  Synchronous. */
rs_status rs_diag_tc_contract(int32_t RP, int32_t rows, const double* v, const double* W,
                              const double* D, double* X, double* Xd);

#ifdef __cplusplus
}
#endif
#endif /* RS_H_ */
