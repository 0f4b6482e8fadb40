/*
 * libwd: Wilson-Dirac operator, its even-odd Schur form and the CGNR solve
 * on one GB300 GPU (sm_103a).
 *
 * The operation (Barthou et al., arXiv:1401.2039):
 *   D = I - kappa * H                                       Fig. "dirac", mu = 0
 *   (H psi)(x) = sum_mu [ (1 - gamma_mu) U_mu(x)       phi_mu  psi(x+mu)
 *                        + (1 + gamma_mu) U_mu(x-mu)^dag phi_mu* psi(x-mu) ]
 * with 4x4 gamma matrices in the DeGrand-Rossi basis (the paper fixes only
 * their algebra, Fig. "id"), 3x3 SU(3) links U (U[s x d]^dag = U[(s+d) x -d],
 * Fig. "id") and a complex boundary phase phi_mu applied to hops that wrap
 * around the lattice in direction mu (conjugated on backward hops; the
 * paper's isPeriodic(L) = true is phi = 1).
 *   Schur operator on parity p (Alg. "schur", D11 = D22 = I):
 *     Mhat_p = I - kappa^2 P_p H P_q^t P_q H P_p^t,  q = 1 - p
 *   Solve (goal "xx = Dirac^-1 bb" with templates "CGNR schur"):
 *     bhat_p = b_p + kappa P_p H b_q; CGNR (Alg. "CGNR") on Mhat_p x_p = bhat_p;
 *     x_q = b_q + kappa P_q H x_p.
 *
 * Canonical layout of every array crossing this boundary (complex128 =
 * two doubles, re then im), all of them DEVICE pointers unless a function
 * says otherwise:
 *   site index  lex = ((t*Lz + z)*Ly + y)*Lx + x;  parity (x+y+z+t) % 2
 *   spinor      [V][3 colour][4 spin] complex128   (full lattice, V sites)
 *   half spinor [V/2][3][4] complex128, entry lex/2 of each site of one parity
 *   gauge field [V][4 mu][3 row][3 col] complex128, mu = x, y, z, t
 * The caller owns every array it passes; calls never keep a pointer to
 * them.  The operator handle owns its packed copies (structure-of-arrays,
 * even-odd ordered, in its storage precision) and all workspace, allocated
 * by wd_op_create; apply and solve calls allocate nothing.
 *
 * Streams: every call is ordered after the work already queued on the
 * stream given to wd_op_create (NULL = the legacy default stream) and the
 * work it queues completes before later work on that stream.  Calls on one
 * handle must not run concurrently from several host threads.
 *
 * Errors: every int-returning call returns a wd_status; none aborts or
 * exits.  wd_last_error() describes the last failure of the calling thread.
 */
#ifndef WD_H
#define WD_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wd_op wd_op;

typedef enum {
    WD_OK = 0,
    WD_ERR_ARG = 1,            /* null pointer, bad parity/flag/precision/recon   */
    WD_ERR_DIMS = 2,           /* a lattice extent odd or < 2, or too large       */
    WD_ERR_CUDA = 3,           /* a CUDA runtime call failed                      */
    WD_ERR_NOMEM = 4,          /* device allocation failed                        */
    WD_ERR_NOT_CONVERGED = 5,  /* solver reached maxiter                          */
    WD_ERR_BREAKDOWN = 6,      /* NaN/Inf or a zero denominator in the solver     */
    WD_ERR_TIMEOUT = 7,        /* a bounded device wait gave up                   */
    WD_ERR_STATE = 8           /* call out of order (e.g. no gauge field loaded)  */
} wd_status;

typedef enum { WD_F64 = 0, WD_F32 = 1, WD_F16 = 2, WD_BF16 = 3 } wd_prec;

/* Create an operator for a Lx x Ly x Lz x Lt lattice.
 *   dims   host int[4] {Lx, Ly, Lz, Lt}; every extent even and >= 2
 *   kappa  hopping parameter (any real; kappa = 0 gives D = I)
 *   phase  host double[8]: (re, im) of phi_mu for mu = x, y, z, t
 *   prec   storage precision of the operator applications and of the
 *          inner solver iterations (WD_F64: plain FP64 throughout;
 *          WD_F32/F16/BF16: low-precision storage, FP32 arithmetic,
 *          FP64 reliable updates in wd_solve_cg)
 *   recon  18 (full links) or 12 (two rows stored, third row rebuilt as
 *          conj(row0 x row1), valid for SU(3) links)
 *   stream cudaStream_t to order work on, or NULL for the legacy stream
 * Allocates every device buffer the handle will need. */
int wd_op_create(wd_op **op, const int dims[4], double kappa, const double phase[8],
                 int prec, int recon, void *stream);
void wd_op_destroy(wd_op *op);

/* Load (copy, pack, convert) the gauge field; U is a device pointer in the
 * canonical [V][4][3][3] complex128 layout.  With recon = 12 the links must
 * be SU(3) for the results to match the 18-real operator. */
int wd_op_set_gauge(wd_op *op, const double *U);

/* out = D in (dagger: D^dag in), full lattice, canonical spinors (Fig. "dirac"). */
int wd_apply(wd_op *op, double *out, const double *in, int dagger);

/* out = Mhat_p in (dagger: Mhat_p^dag in) on half-lattice spinors of parity p
 * (Alg. "schur": D22 - D21 D11^-1 D12 for p = 1). */
int wd_apply_eo(wd_op *op, double *out, const double *in, int parity, int dagger);

/* out = Mhat_p in (dagger: Mhat_p^dag in) as wd_apply_eo, but evaluated in
 * the handle's residual arithmetic -- the arithmetic of the reliable updates
 * (native FP64, or double-float for mixed-precision handles, selected with
 * wd_op_set_residual_precision) on the FP64-side 18-real copy of the links.
 * Same layout, ownership and errors as wd_apply_eo.  Lets a caller check
 * residuals, or the double-float arithmetic, against an FP64 reference. */
int wd_apply_eo_residual(wd_op *op, double *out, const double *in, int parity, int dagger);
/* As wd_apply_eo_residual in the arithmetic of the early refreshes of a
 * mixed-precision solve (those whose residual is still above 1e-5 of ||b||):
 * the double-float fields and links read in FP32 arithmetic, each
 * double-float rounded to one float on load (relative rounding ~1e-7).
 * Handles with FP64 residuals have no early form: the call is
 * wd_apply_eo_residual. */
int wd_apply_eo_residual_early(wd_op *op, double *out, const double *in, int parity,
                               int dagger);

/* out = P_p H P_q^t in (dagger: the same with H^dag): the hopping term from
 * parity q = 1 - p onto parity p, half-lattice canonical spinors. */
int wd_dslash_eo(wd_op *op, double *out, const double *in, int out_parity, int dagger);

typedef struct {
    int iters;               /* inner CGNR iterations                             */
    int reliable_updates;    /* FP64 residual recomputations                      */
    double true_rel_resid;   /* ||b - D x|| / ||b|| in FP64 on the full lattice    */
    double seconds;          /* host wall time of the call                         */
    double dslash_lo;        /* hopping-term applications in storage precision     */
    double dslash_hi;        /* hopping-term applications in FP64                  */
    double bytes;            /* algorithmic device bytes moved by the solve        */
    double launches;         /* kernels launched (directly or inside CUDA graphs)  */
    int restarts;            /* Krylov restarts after a stagnating residual        */
} wd_solve_info;

/* Solve D x = b (goal "xx = Dirac^-1 bb", templates "CGNR schur") to
 * ||b - D x|| / ||b|| <= tol, judged by an FP64 true residual.
 *   x       device, full canonical spinor; on entry its parity-p part is the
 *           initial guess (zeros for none), on exit the solution
 *   b       device, full canonical spinor
 *   parity  the parity CGNR works on (1 = odd, as in Alg. "schur")
 *   info    may be NULL
 * Returns WD_OK, WD_ERR_NOT_CONVERGED (x holds the last iterate) or
 * WD_ERR_BREAKDOWN.  Blocks the calling thread until the solve is done. */
int wd_solve_cg(wd_op *op, double *x, const double *b, double tol, int maxiter,
                int parity, wd_solve_info *info);

/* Reliable-update parameters of the mixed-precision solve (ignored for
 * WD_F64): the FP64 residual is recomputed whenever the iterated residual
 * has fallen by ru_delta (0 < ru_delta < 1; default 0.01 for WD_F32, 0.1
 * for WD_F16, 0.3 for WD_BF16) since the last
 * recomputation, and the Krylov direction restarts when the iterated residual
 * has not improved for stall_iters iterations (default 200). */
int wd_op_set_solver(wd_op *op, double ru_delta, int stall_iters);

/* How the mixed-precision solve recovers FP64 accuracy (ignored for WD_F64;
 * not in the paper, which runs CGNR in one precision):
 *   WD_RECOVER_RELIABLE (default)  reliable updates (Clark et al. 2010): when
 *       the iterated residual has fallen by ru_delta (wd_op_set_solver) the
 *       inner solution is folded into the FP64 one, the residual is
 *       recomputed in the residual arithmetic and the inner CGNR goes on with
 *       its Krylov direction rescaled to the new residual;
 *   WD_RECOVER_DEFECT  defect correction (iterative refinement): each outer
 *       step computes r = bhat - Mhat x in the residual arithmetic, solves
 *       Mhat e = r with an inner CGNR (Alg. "CGNR") in the storage precision
 *       started from e = 0 in a fresh Krylov space until its iterated
 *       residual has fallen by inner_tol (0 < inner_tol < 1, default 0.1),
 *       and adds e to the FP64 x.
 * Both stop on the same FP64 true residual; wd_solve_info.reliable_updates
 * counts the residual recomputations (outer steps) of either.
 * WD_ERR_ARG for another mode or an inner_tol outside (0, 1). */
typedef enum { WD_RECOVER_RELIABLE = 0, WD_RECOVER_DEFECT = 1 } wd_recovery;
int wd_op_set_recovery(wd_op *op, int mode, double inner_tol);
/* The handle's recovery mode (-1 for a null handle) and, if inner_tol is not
 * NULL, its defect-correction inner tolerance. */
int wd_op_recovery(const wd_op *op, double *inner_tol);

/* Arithmetic of the residual recomputations of the reliable updates, of the
 * Schur preparation and reconstruction and of the final true residual for
 * WD_F32/WD_F16/WD_BF16 operators: mode 0 = native FP64, mode 1 (default) =
 * double-float (each real the unevaluated sum of two FP32 numbers, a 48-bit
 * significand, run on the FP32 pipes; GB300's FP64 rate is a small fraction
 * of its FP32 rate).  Either form keeps ||b - D x|| accurate far below the
 * 1e-10 relative residuals the solver is used for.  WD_F64 operators always
 * use FP64 (mode 1 is rejected).  Not in the paper. */
int wd_op_set_residual_precision(wd_op *op, int mode);

/* Twisted mass (Fig. "dirac": D = 1 + 2 i kappa mu gamma5 - kappa H; the
 * handle starts with mu = 0, the Wilson operator).  With mu != 0 every
 * operator call of the handle includes the term: wd_apply applies D (the
 * adjoint flips the sign of mu), wd_apply_eo and wd_apply_eo_residual apply
 * Mhat_p = A - kappa^2 H_pq A^-1 H_qp with A = 1 + 2 i kappa mu gamma5 (the
 * diagonal block D11 of Alg. "schur", inverted site by site), and
 * wd_solve_cg solves D x = b through bhat_p = b_p + kappa H_pq A^-1 b_q and
 * x_q = A^-1 (b_q + kappa H_qp x_p).  wd_dslash_eo stays the bare hopping
 * term; wd_apply_eo_noalloc and batches (wd_batch_*) have no twisted mass
 * (a batch over a twisted handle returns WD_ERR_ARG).  mu must be finite
 * (WD_ERR_ARG otherwise). */
int wd_op_set_twisted_mass(wd_op *op, double mu);
/* The handle's mu (0 for a null handle). */
double wd_op_twisted_mass(const wd_op *op);

/* The same solve with x and b in HOST memory (pageable or pinned); the
 * host<->device copies go through buffers the handle owns.  b goes up in
 * eight slabs of time slices, and the solve's preparation starts on each
 * slab as it lands; x comes down as soon as it is complete, while the final
 * true residual is computed.  The call returns when x_host holds x. */
int wd_solve_cg_host(wd_op *op, double *x_host, const double *b_host, double tol,
                     int maxiter, int parity, wd_solve_info *info);
/* As wd_solve_cg_host from the initial guess x = 0: x_host is output only
 * and is not read, so only b crosses to the device (and x back). */
int wd_solve_cg_host_zero_guess(wd_op *op, double *x_host, const double *b_host, double tol,
                                int maxiter, int parity, wd_solve_info *info);
/* A stream of n host-memory solves D x_k = b_k (k = 0 .. n-1), each from the
 * initial guess 0, one after another on the handle: b_{k+1} goes up (into a
 * second device staging buffer, allocated at the first call: 384 x Vh bytes)
 * while solve k runs, and x_k comes down while solve k+1 runs, so that a
 * serving loop pays about one device solve per source.  x_host[k], b_host[k]
 * as in wd_solve_cg_host_zero_guess (the x_host[k] must not overlap any
 * b_host[j]; entries may repeat: a repeated x_host holds the last of its
 * solutions, a repeated b_host is read again); infos (optional) receives n
 * entries, seconds being each solve's host time (from queueing the next
 * source's upload to the solve's end).  Every solution is bitwise the one wd_solve_cg_host_zero_guess
 * gives.  The call returns when all x_host[k] hold their solutions, or at the
 * first failing solve (its code; later ones are not run).  n = 0 does
 * nothing; n < 0 or a null pointer among the first n is WD_ERR_ARG. */
int wd_solve_cg_host_stream(wd_op *op, int n, double *const *x_host,
                            const double *const *b_host, double tol, int maxiter, int parity,
                            wd_solve_info *infos);

/* ---------------------------------------------------------------------------
 * Batches: several operators (lattices of any size, one storage precision
 * and link format, FP64/FP32/FP16) with nrhs[k] right-hand sides each, at
 * most 8 operators and 64 systems.  A batch owns the fields of all its
 * systems (right-hand-side index innermost, so the links of a site are read
 * once for all of its right-hand sides) and advances every system in
 * lockstep with persistent kernels that walk a table of tiles over all
 * lattices; each system keeps its own CGNR scalars, residual refreshes
 * (reliable updates, or the outer steps of defect correction: the recovery
 * mode and tolerances of the first operator apply to every system) are
 * taken together, and converged systems are frozen.  The operators must
 * outlive the batch.  Not in the paper: it batches the paper's solve (goal
 * with templates "CGNR schur") over many right-hand sides and lattices. */
typedef struct wd_batch wd_batch;
int wd_batch_create(wd_batch **bt, wd_op *const *ops, const int *nrhs, int nops);
void wd_batch_destroy(wd_batch *bt);
/* out[k], in[k]: device, [nrhs[k]][V_k/2][3][4] complex128, hopping term
 * P_p H P_q^t of every system (storage precision of the operators). */
int wd_batch_dslash(wd_batch *bt, double *const *out, const double *const *in, int out_parity,
                    int dagger);
/* The same on the batch's resident fields (last inputs of wd_batch_dslash). */
int wd_batch_dslash_resident(wd_batch *bt, int out_parity, int dagger);
/* Launch configuration of the batched hopping term picked by the autotuner
 * when the batch was created (FP32/FP16 storage; every candidate is timed on
 * the batch's own lattices and right-hand sides): variant 0 = the plain hop,
 * 1 = the xpay hop with the fused per-system norms that ends each Schur
 * operator of the lockstep CGNR.  There are 9 candidates: 0-4 take one
 * (site, rhs) item per thread, 5-8 two (rhs r and r + 1 of one site, FP32
 * storage with an even number of right-hand sides in every problem; 0 us
 * where they do not apply).  us (optional, n entries) receives each
 * candidate's microseconds per launch; block (threads per block), min_blocks
 * (resident blocks per SM the register cap is set for) and grid (the
 * persistent grid launched: the kernel's resident capacity on this GPU, at
 * most the tile count) describe the chosen one.  Returns its index, or -1
 * for a null batch or another variant.  WD_BATCH_CFG=k forces candidate k
 * (where it applies), WD_TUNE=0 keeps candidate 0. */
int wd_batch_tuning(const wd_batch *bt, int variant, double *us, int n, int *block,
                    int *min_blocks, int *grid);
/* x[k] (in: initial guesses or zeros, out: solutions), b[k]: device,
 * [nrhs[k]][V_k][3][4] complex128; info: sum(nrhs) entries or NULL, in
 * system order (operator 0's right-hand sides first). */
int wd_batch_solve(wd_batch *bt, double *const *x, const double *const *b, double tol,
                   int maxiter, int parity, wd_solve_info *info);
const char *wd_batch_last_error(void);
/* One-call form of the batched solve: wd_batch_create, wd_batch_solve and
 * wd_batch_destroy in one (the same arguments, order and errors; the error
 * text is in wd_batch_last_error).  It allocates and frees the batch's
 * fields on every call; repeated solves should keep a wd_batch instead. */
int wd_solve_cg_multi(wd_op *const *ops, int nops, double *const *x, const double *const *b,
                      const int *nrhs, double tol, int maxiter, int parity,
                      wd_solve_info *info);

/* Resident fields for timing the hopping term alone: slot 0 and 1 are two
 * half-lattice spinors the handle owns, in its internal layout and storage
 * precision.  wd_field_load packs a canonical half spinor (device) into a
 * slot, wd_field_store unpacks it, wd_dslash_resident computes
 * slot[1 - in_slot] = P_p H P_q^t slot[in_slot] with no layout conversion. */
int wd_field_load(wd_op *op, int slot, const double *half_in);
int wd_field_store(wd_op *op, int slot, double *half_out);
int wd_dslash_resident(wd_op *op, int in_slot, int out_parity, int dagger);

/* Launch configuration of the hopping term picked by the autotuner when the
 * gauge field was loaded.  hi = 0: the storage-precision kernel; hi = 1: the
 * residual-arithmetic (FP64 or double-float) kernel of the reliable updates;
 * hi = 2: the storage-precision kernel with the xpay epilogue and fused norm
 * that ends each Schur operator of the CGNR iteration (tuned on its own: its
 * register demand differs).  us (optional, n entries) receives the
 * measured microseconds per launch of every candidate (0 for a candidate
 * that was not timed: link staging applies to FP16/BF16 storage only, and
 * entries past the candidate count); block, min_blocks, sites_per_thread and
 * staged (optional; staged = 1: the link records of the eight hops are copied
 * into shared memory at kernel start and the neighbour spinors are loaded two
 * hops ahead; staged = 2: the same with the spinors three hops ahead)
 * describe the chosen one.  Returns its
 * index, or -1 for a null handle.  Setting WD_DSLASH_CFG=k in the
 * environment forces candidate k, WD_TUNE=0 keeps candidate 0. */
int wd_dslash_tuning(const wd_op *op, int hi, double *us, int n, int *block, int *min_blocks,
                     int *sites_per_thread, int *staged);

/* Stream the handle queues its work on (a cudaStream_t). */
void *wd_op_stream(wd_op *op);

/* Number of sites of one parity, V/2 (0 for a null handle). */
long wd_op_half_volume(const wd_op *op);

/* Algorithmic (compulsory) bytes of one single-parity hopping-term launch in
 * the handle's storage precision: Vh * (24 in + 24 out + 8 links * recon)
 * reals. */
double wd_dslash_bytes(const wd_op *op);

const char *wd_status_string(int status);
const char *wd_last_error(void);

/* ---------------------------------------------------------------------------
 * Schur operator for callers that cannot allocate device memory.
 *
 * The paper has no counterpart: this is a deployment variant of
 * wd_apply_eo.  Callers that cannot call cudaMalloc (code running while a
 * host framework captures its stream into a CUDA graph, plug-ins whose host
 * application owns all device memory through its own pool, real-time paths
 * that must not enter the driver's allocator) cannot create a wd_op, which
 * allocates.  This entry point needs no handle and allocates nothing: it
 * reads the caller's canonical FP64 arrays directly and keeps its one
 * intermediate field in a fixed device array inside libwd (12,582,912
 * bytes, held on every GPU where this entry point has been called, from the
 * first call until the process exits).
 *
 *   out     device, [V/2][3][4] complex128, parity `parity`; must not overlap in
 *   in      device, [V/2][3][4] complex128, parity `parity`
 *   U       device, [V][4][3][3] complex128 (canonical gauge field)
 *   dims, kappa, phase, parity, dagger: as for wd_op_create / wd_apply_eo
 *   stream  cudaStream_t the two kernels are queued on (NULL = legacy)
 * out = Mhat_p in (dagger: Mhat_p^dag in), FP64 throughout, asynchronous.
 *
 * Limits and sharing: V/2 must not exceed WD_NOALLOC_MAX_VH (else
 * WD_ERR_DIMS, nothing queued).  Every call shares the one device array,
 * which keeps the last call's contents; calls that overlap on the GPU
 * (different streams or host threads) race on it and must be serialised by
 * the caller.  The first call on each device loads the entry point's kernels
 * there and looks up the array's device address (cudaGetSymbolAddress, with
 * that device current); make that first call before any stream capture
 * begins.  Extents whose product exceeds the maximum are rejected before
 * any arithmetic can overflow.  Errors are described by
 * wd_noalloc_last_error().
 */
#define WD_NOALLOC_MAX_VH 65536
int wd_apply_eo_noalloc(double *out, const double *in, const double *U, const int dims[4],
                        double kappa, const double phase[8], int parity, int dagger,
                        void *stream);
const char *wd_noalloc_last_error(void);

/* ---------------------------------------------------------------------------
 * Learned preconditioner (not in the paper): a linear, gauge-equivariant
 * parallel-transport convolution network (Lehner & Wettig, arXiv:2302.05419)
 * that maps one spinor field to one through layers of channels[0..nlayers]
 * (channels[0] = channels[nlayers] = 1):
 *   out_c'(x) = sum_c sum_{k=0..8} W[c', c, k] (T_k in_c)(x),
 * W[c', c, k] complex 4x4 spin matrices, T_0 = 1,
 * T_{1+mu} psi(x) = U_mu(x) phi_mu psi(x+mu), T_{5+mu} psi(x) =
 * U_mu(x-mu)^dag phi_mu^* psi(x-mu) (phases on hops that wrap).  The channel
 * mixing runs on the tensor cores (BF16 operands, FP32 accumulation).
 * Every call is ordered after the work queued on the stream given at
 * creation and completes before later work on it.
 * Weights cross the boundary as one device complex128 vector, layers in
 * order, each [C_out][C_in][9][4][4]; gradients use the same layout packed as
 * dL/dRe W + i dL/dIm W.  Spinors are device canonical [V][3][4] complex128.
 */
typedef struct wd_ptc wd_ptc;
int wd_ptc_create(wd_ptc **net, const int dims[4], const double phase[8], int nlayers,
                  const int *channels, void *stream);   /* stream as for wd_op_create */
void wd_ptc_destroy(wd_ptc *net);
int wd_ptc_set_gauge(wd_ptc *net, const double *U);       /* canonical [V][4][3][3] */
long wd_ptc_weight_count(const wd_ptc *net);              /* complex weights in total */
int wd_ptc_set_weights(wd_ptc *net, const double *W);
int wd_ptc_get_weights(wd_ptc *net, double *W);
int wd_ptc_apply(wd_ptc *net, double *y, const double *r);  /* y = N(r), synchronous */
/* How wd_ptc_apply runs a layer with 16 input and 16 or 1 output channels:
 * on = 1 (default) as one fused kernel that computes the transports straight
 * into the tensor cores' shared-memory operand tiles (nothing of the
 * gathered operand goes to HBM); on = 0 as a gather of the transported
 * operand into device memory followed by the tensor-core GEMM (the form
 * training always uses: its weight gradient needs that operand).  The two
 * differ only in the order of the FP32 accumulation. */
int wd_ptc_set_fused(wd_ptc *net, int on);
/* Loss L = sum_i ||N(r_i) - e_i||^2 / ||e_i||^2 over nsamples fields r, e
 * ([nsamples][V][3][4]) and its gradient (grad: device, weight layout, or NULL). */
int wd_ptc_loss_grad(wd_ptc *net, const double *r, const double *e, int nsamples,
                     double *loss, double *grad);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) with learning rate lr on
 * the same loss; *loss receives the loss before the step. */
int wd_ptc_train_step(wd_ptc *net, const double *r, const double *e, int nsamples, double lr,
                      double *loss);
/* The network's tensor-core GEMM alone, D = A B^T (A [M][K], B [N][K] BF16,
 * D [M][N] FP32, device; M % 128 == 0, N % 16 == 0, K % 64 == 0). */
int wd_tc_gemm_bf16(wd_ptc *net, const void *A, const void *B, float *D, long M, int N, int K);
/* The transposed tensor-core GEMM of the weight gradient alone, D = A^T B
 * (A [R][M], B [R][N] BF16 row-major, D [M][N] FP32, device; the reduction
 * over the R rows is split over CTAs and summed in a fixed order;
 * R % 64 == 0, M % 128 == 0, N % 16 == 0). */
int wd_tc_gemm_bf16_tn(wd_ptc *net, const void *A, const void *B, float *D, long R, int M, int N);
/* Bounded waits of the network's tensor-core GEMMs: every wait of a GEMM on
 * its MMAs polls at most `polls` times (default 2^26) before the kernel gives
 * up, lets the MMAs it issued drain, frees its tensor memory and the call
 * returns WD_ERR_TIMEOUT.  withhold_mma = 1 (for tests of that path) makes
 * the GEMMs issue no MMA at all, so that their first wait runs out with
 * nothing in flight.  WD_ERR_ARG for polls = 0 or withhold_mma not 0/1. */
int wd_ptc_set_wait_limit(wd_ptc *net, unsigned polls, int withhold_mma);
const char *wd_ptc_last_error(void);

/* Flexible GCR(nkrylov) on the full system D x = b (not in the paper), with
 * the network as right preconditioner (net may be NULL: plain GCR).  w = D z
 * uses op_lo (any storage precision); the residual is recomputed with op_hi
 * (a WD_F64 operator on the same lattice) at every restart, and the solve
 * stops when ||b - D x|| / ||b|| <= tol by that FP64 residual.  x, b: device
 * canonical [V][3][4] complex128.  info->iters counts preconditioned
 * directions, info->reliable_updates restarts.  The handle owns its basis
 * (2 nkrylov + 3 fields); the operators and the network must outlive it. */
typedef struct wd_fgcr wd_fgcr;
int wd_fgcr_create(wd_fgcr **solver, wd_op *op_lo, wd_op *op_hi, wd_ptc *net, int nkrylov);
void wd_fgcr_destroy(wd_fgcr *solver);
int wd_fgcr_solve(wd_fgcr *solver, double *x, const double *b, double tol, int maxiter,
                  wd_solve_info *info);
const char *wd_fgcr_last_error(void);

/* The other solvers of the paper's solver comparison (Sec. 5, Fig.
 * "algosxp": CGNR, CRNE, MCR1, MCR2 on the Schur system), which the paper
 * names without defining; textbook readings:
 *   WD_KRYLOV_CGNR  Alg. "CGNR" (as wd_solve_cg with WD_F64, host-driven)
 *   WD_KRYLOV_CRNE  conjugate residual (Saad, Iterative Methods for Sparse
 *                   Linear Systems, Alg. 6.20) on Mhat Mhat^dag y = bhat,
 *                   x = Mhat^dag y; two operator applications per iteration
 *   WD_KRYLOV_MCR1  conjugate residual on the Hermitian indefinite
 *                   gamma5 Mhat x = gamma5 bhat, B p formed by the operator
 *                   (two applications per iteration)
 *   WD_KRYLOV_MCR2  the same with B p updated by recurrence (one application)
 * MCR relies on gamma5-hermiticity (Mhat^dag = gamma5 Mhat gamma5), which a
 * twisted mass breaks: a solve with mu != 0 returns WD_ERR_ARG for MCR1/2.
 *
 * wd_krylov_create: op must be a WD_F64 operator (the methods run in FP64);
 * the handle owns 9 half-lattice FP64 fields and keeps a pointer to op,
 * which must outlive it.  wd_krylov_solve: the same arguments and layout as
 * wd_solve_cg (x, b device canonical [V][3][4] complex128; the parity-p part
 * of x on entry is the initial guess), the same Schur preparation and
 * reconstruction (with the twisted mass of op), and x is accepted only on
 * the FP64 true residual ||b - D x|| / ||b|| <= tol; when the recursive
 * residual met the target but the true one does not, the method restarts
 * from x.  info->iters counts iterations, info->reliable_updates true-
 * residual checks, info->dslash_hi hopping terms.  Returns WD_OK,
 * WD_ERR_NOT_CONVERGED, WD_ERR_BREAKDOWN ((r|B r) or |B p| zero, or a
 * non-finite residual), WD_ERR_ARG or WD_ERR_STATE (no gauge field);
 * blocks until done. */
typedef enum {
    WD_KRYLOV_CGNR = 0,
    WD_KRYLOV_CRNE = 1,
    WD_KRYLOV_MCR1 = 2,
    WD_KRYLOV_MCR2 = 3
} wd_krylov_method;
typedef struct wd_krylov wd_krylov;
int wd_krylov_create(wd_krylov **solver, wd_op *op, int method);
void wd_krylov_destroy(wd_krylov *solver);
int wd_krylov_solve(wd_krylov *solver, double *x, const double *b, double tol, int maxiter,
                    int parity, wd_solve_info *info);
const char *wd_krylov_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* WD_H */
