/*
 * sailfish_gb300.h -- C ABI of the GB300 fast Poisson solver library
 * (libsailfish_gb300.so).
 *
 * The library solves  lap(psi) = rhs_scale * f  on a rectangular 1D, 2D or 3D
 * grid with the spectral method of SailFFish (Saverin, arXiv 2301.01145):
 * forward transform, point-wise multiply by the eigenvalues or by the
 * transformed Green's function, optional spectral operator, inverse
 * transform (Sec. 2.4, "Calculating and Retrieving the Solution").
 *
 * Conventions used by every call
 *  - Arrays are row-major [component][z][y][x] (x fastest), 2D: [component][y][x],
 *    1D: [component][x].
 *  - Element type is float (SF_F32) or double (SF_F64), chosen per plan.
 *  - Device pointers must be CUDA device (or managed) memory on the current
 *    device, 16-byte aligned.  Host pointers are only accepted by
 *    sf_solve_host and sf_solve_host_many.  The caller owns every buffer it passes; the library
 *    records pointers (no copies) and reads/writes them when the enqueued work
 *    runs on the plan's stream, so buffers must stay alive until then.
 *  - Every call returns an sf_status; no C++ exception crosses the ABI.
 *    sf_last_error() gives a thread-local human-readable detail string.
 *  - Work is asynchronous on the plan's CUDA stream unless stated otherwise.
 *    Device-side failures (a scheduler wait that gave up, a CUDA error) are
 *    reported by sf_sync() or by the next call on the plan.
 *  - No call is thread-safe on the same plan; distinct plans are independent.
 */
#ifndef SAILFISH_GB300_H
#define SAILFISH_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sf_plan_s *sf_plan; /* opaque; created and owned by the library */

typedef enum {
  SF_OK = 0,
  SF_ERR_ARG = -1,         /* invalid argument or descriptor                         */
  SF_ERR_UNSUPPORTED = -2, /* valid option combination that this library lacks       */
  SF_ERR_CUDA = -3,        /* a CUDA runtime call failed (detail in sf_last_error)   */
  SF_ERR_OOM = -4,         /* device allocation failed                               */
  SF_ERR_STATE = -5,       /* call out of order (e.g. solve without a source)        */
  SF_ERR_TIMEOUT = -6,     /* a bounded device-side wait in the scheduler gave up    */
  SF_ERR_CORRUPT = -7      /* SF_FLAG_DEBUG_CHECKS: a workspace guard band was overwritten */
} sf_status;

/* Boundary type of an axis (Sec. 2.4.1 solver types; Sec. 2.5 bounded, 2.6 unbounded). */
typedef enum { SF_BC_PERIODIC = 0, SF_BC_DIRICHLET = 1, SF_BC_NEUMANN = 2, SF_BC_UNBOUNDED = 3 } sf_bc;

/* Grid type (Sec. 2.4.2, Eq. gridpos): REGULAR = cell-boundary nodes, STAGGERED = cell centres. */
typedef enum { SF_GRID_REGULAR = 0, SF_GRID_STAGGERED = 1 } sf_grid;

/* Spectral operator applied to psi after the convolution (Sec. 2.4.3, Eq. ft_sd). */
typedef enum { SF_OP_NONE = 0, SF_OP_GRAD = 1, SF_OP_DIV = 2, SF_OP_CURL = 3, SF_OP_NABLA = 4 } sf_op;

/* Eigenvalue type for bounded axes (Sec. 2.5.2, Table 1). */
typedef enum { SF_EIG_PS = 0, SF_EIG_FD2 = 1 } sf_eig;

/* Unbounded kernels (Sec. 2.6.2): Gaussian regularisation of order 2 to 10 (2D, 3D).
 * G_P = G2 + sum_{j=1}^{P/2-1} sigma^{2j} / (2^j j!) (-lap)^{j-1} zeta_sigma, the
 * kernel whose smoothing has the transform exp(-(k sigma)^2/2) times the Taylor
 * series of exp(+(k sigma)^2/2) cut below order P (error O((k sigma)^P)). */
/* SF_GREEN_SPECTRAL (1D, 2D and 3D; the only 1D kernel, Sec. 4.3): the sharp
 * spectral cut-off G^(k) = 1/k^2 for |k| <= kc = pi / max_axis h, zero beyond,
 * i.e. G(r) = Si(kc r) / (2 pi^2 r) in 3D,
 * G(r) = (ln(kc / 2) + gamma - F(kc r)) / (2 pi), F(x) = int_0^x (1 - J0(t)) / t dt
 * in 2D (constant chosen so that G + ln(r) / (2 pi) -> 0, the far field of the
 * 2D free-space kernel -ln(r) / (2 pi)), and
 * G(x) = -(|x| Si(kc |x|) + cos(kc x) / kc) / pi in 1D (constant chosen so that
 * G + |x|/2 -> 0, the far field of -|x|/2); green_sigma is not used. */
typedef enum {
  SF_GREEN_G2 = 0, SF_GREEN_G4 = 1, SF_GREEN_G6 = 2, SF_GREEN_G8 = 3, SF_GREEN_G10 = 4, SF_GREEN_SPECTRAL = 5
} sf_green;

typedef enum { SF_F32 = 0, SF_F64 = 1 } sf_prec;

/* Plan flags (sf_plan_desc.flags). */
#define SF_FLAG_UNFUSED 1u /* one kernel launch per pass instead of one persistent launch */
#define SF_FLAG_GENERIC 2u /* always use the general shared-memory FFT engine (no register fast path) */
/* Debug checks: every device buffer of the plan (workspace and tables) is
 * allocated with a 4 KB guard band on each side, filled with the byte 0xA5;
 * sf_sync scans the bands after the stream drains and returns SF_ERR_CORRUPT if
 * any byte changed (an out-of-range write by the library).  The slack between a
 * buffer's end and the next 256-byte boundary is not guarded.  Costs one 4 KB
 * device-to-host copy per band on every sf_sync. */
#define SF_FLAG_DEBUG_CHECKS 4u

/*
 * Problem description (Sec. 2.4 solver options, Sec. 2.5.1 Table 1).
 *   dim        1, 2 or 3 (Sec. 2.4: the 1D / 2D / 3D solver classes).
 *   n[a]       cell count N_c per axis a = x, y, z (axes a >= dim ignored).  Every
 *              FFT length used (N_c for periodic, 4 N_c for an axis with a
 *              Dirichlet and a Neumann face, 2 N_c otherwise) must be of the
 *              form 2^p or 3*2^p and lie in [4, 2048]; 2 <= N_c <= 2048
 *              (N_c >= 3 for regular Dirichlet on both faces).  An unbounded
 *              axis on the regular grid (N_c + 1 nodes) is padded to the
 *              smallest 2^p or 3*2^p >= 2 N_c + 1.
 *   lo, hi     domain bounds X_l < X_u per axis (finite, finite difference).
 *   bc[a][s]   boundary type of axis a on its lower (s = 0) and upper (s = 1)
 *              face.  The faces of an axis agree, or one is Dirichlet and the
 *              other Neumann: that axis is then transformed in the quarter-wave
 *              sine (Dirichlet lower) or cosine (Neumann lower) basis, modes
 *              k + 1/2 (FFTW's RODFT01 / RODFT11 and REDFT01 / REDFT11 on the
 *              regular / staggered grid), the paper's stated next step beyond
 *              its uniform boundaries (Sec. 2.4.1).  On a regular grid a
 *              Dirichlet face node is filled from the face data and a Neumann
 *              face node is solved for.  Either every axis is
 *              periodic/unbounded, or every axis is Dirichlet/Neumann.
 *              Semi-unbounded (2D, 3D): exactly one unbounded axis, the others
 *              periodic.  Per periodic mode, kappa^2 = -(sum of the periodic
 *              axes' eigenvalues, PS or FD2) and the unbounded axis carries
 *              the free-space kernel of -(d^2/dz^2 - kappa^2),
 *              exp(-kappa |z|) / (2 kappa), or -|z| / 2 for kappa = 0,
 *              point-sampled and summed by doubling that axis (the paper names
 *              such domains as its next step without their kernels, Sec. 2.6,
 *              Sec. 6); green and green_sigma are not used.  Two unbounded axes
 *              with a periodic one return SF_ERR_UNSUPPORTED.
 *   grid       REGULAR (N_c + 1 nodes per axis) or STAGGERED (N_c cell centres).
 *   eig        PS or FD2 (bounded and periodic axes; ignored on unbounded axes).
 *   op         spectral operator on psi.  On Dirichlet / Neumann axes a
 *              derivative differentiates the axis's sine / cosine series
 *              (sine <-> cosine) and is evaluated at every node (zero where the
 *              series vanishes).
 *              GRAD: ncomp 1 -> dim outputs.  DIV: ncomp = dim -> 1 output.
 *              CURL: 3D ncomp 3 -> 3 outputs; 2D ncomp 1 -> 2 outputs; not 1D.
 *              NABLA: ncomp -> ncomp outputs.  In 1D, GRAD and DIV are d/dx.
 *   green      kernel for unbounded solves; green_sigma its Gaussian width
 *              (positive and finite; ignored by SF_GREEN_SPECTRAL).
 *   ncomp      number of field components solved together (1..3).
 *   prec       arithmetic of the solve (tables are always built in FP64).
 *   rhs_scale  the plan solves lap(psi) = rhs_scale * f.
 *   flags      SF_FLAG_* bits, 0 by default; any other bit is SF_ERR_ARG.
 */
typedef struct {
  int32_t dim;
  int32_t n[3];
  double lo[3];
  double hi[3];
  int32_t bc[3][2];
  int32_t grid;
  int32_t eig;
  int32_t op;
  int32_t green;
  double green_sigma;
  int32_t ncomp;
  int32_t prec;
  double rhs_scale;
  uint32_t flags;
  /* tuning knobs (0 = library default), chosen by the autotuner:
   *   tune_radix  largest radix of the general FFT engine (2, 4, 8 or 16)
   *   tune_tile   largest number of packed lines per tile of the general engine (1..16, power of 2)
   *   tune_slab   kx planes per slab of the register fast path's pipeline (>= 1)
   *   tune_lag    slabs between the pipeline's stages (>= 1; ring depth = lag + 2) */
  int32_t tune_radix;
  int32_t tune_tile;
  int32_t tune_slab;
  int32_t tune_lag;
} sf_plan_desc;

/*
 * Array extents per axis (Sec. 2.4.2 "the number of resolved grid positions
 * changes depending on the type of solver"):
 *   periodic, unbounded, staggered Dirichlet/Neumann:  N_c points
 *   regular Dirichlet/Neumann:                         N_c + 1 points
 * For regular Dirichlet axes the two boundary nodes of the source are ignored
 * and those of psi are filled with the face values (0 without face data).
 */

/* Create a plan (Sec. 2.4.4 "Solver Initialization": grid set-up, transform
 * plans, Green's function / eigenvalues, operators).  Allocates the plan's
 * tables and workspace with cudaMalloc on the current device and, for
 * unbounded axes, tabulates G and transforms it in FP64 on the GPU.
 * cuda_stream is a cudaStream_t (NULL = legacy default stream) on which all
 * later work of the plan is enqueued.  On failure *out is NULL. */
sf_status sf_plan_create(sf_plan *out, const sf_plan_desc *d, void *cuda_stream);

/* Change the stream later work is enqueued on. */
sf_status sf_plan_set_stream(sf_plan p, void *cuda_stream);

/* Shapes as [ncomp][z][y][x] (2D: [ncomp][1][y][x], 1D: [ncomp][1][1][x]) of the source (in_shape),
 * of psi (out_shape) and of the operator output (op_shape, all zero when op is
 * NONE), and the bytes of device workspace the plan holds.  Any pointer may be
 * NULL. */
sf_status sf_plan_query(sf_plan p, size_t in_shape[4], size_t out_shape[4], size_t op_shape[4],
                        size_t *workspace_bytes);

/* Paper's Set_Input (Sec. 2.4.5): record the device source f; no copy. */
sf_status sf_set_source(sf_plan p, const void *dev_f);

/* Inhomogeneous boundary data for FD2 solves (Sec. 2.5.2, Sec. 4.2).
 * axis 0..dim-1, side 0 (X_l) or 1 (X_u).  dev_face holds one value per node
 * of the two other axes, row-major with the higher axis first ([z][y] for an x
 * face, [z][x] for a y face, [y][x] for a z face; 2D: [y] or [x]; 1D: one value).
 * Dirichlet: psi on the face; Neumann: d psi / d x_axis on the face.
 * NULL removes the face (homogeneous).  Only for ncomp == 1, FD2, D/N axes. */
sf_status sf_set_boundary(sf_plan p, int axis, int side, const void *dev_face);

/* Paper's Forward_Transform + Convolution + Backward_Transform (Sec. 2.4.5):
 * enqueue the forward transforms, the point-wise multiply, the operator and
 * every inverse transform except the last (x) one, whose output is written
 * by sf_get_output.  Needs a source. */
sf_status sf_solve(sf_plan p);

/* Paper's Get_Output: enqueue the final inverse transform along x fused with
 * the extraction of the unpadded result and the Dirichlet boundary fill,
 * writing psi ([ncomp][...]) and, when op != NONE, the operator output (for
 * first derivatives on Dirichlet / Neumann axes, the inverse y / x passes of
 * each derivative term follow; they read the plan's spectral workspace, so no
 * other solve of the plan may run between sf_solve and this call). */
sf_status sf_get_output(sf_plan p, void *dev_psi, void *dev_op_out);

/* Set_Input + solve + Get_Output in one call (one persistent kernel launch
 * unless SF_FLAG_UNFUSED). */
sf_status sf_execute(sf_plan p, const void *dev_f, void *dev_psi, void *dev_op_out);

/* End-to-end solve on HOST buffers: copies f host->device, solves, copies psi
 * (and the operator output) device->host, all on the plan stream, and waits
 * for completion.  Pinned host memory gives full copy bandwidth.  Uses device
 * staging buffers owned by the plan. */
sf_status sf_solve_host(sf_plan p, const void *host_f, void *host_psi, void *host_op_out);

/* n independent end-to-end solves on HOST buffers, pipelined: host_f[i] is
 * copied host->device on a side stream while solve i-1 runs on the plan
 * stream, and the results of solve i are copied device->host on a second
 * side stream while solve i+1 runs.  Two device staging sets owned by the
 * plan alternate (allocated on first use: 2 x (ncomp + nop) fields).  Returns
 * after every copy has landed.  host_f, host_psi (and host_op_out when
 * op != NONE) are tables of n host pointers laid out as for sf_solve_host;
 * pinned memory gives full copy bandwidth and lets the copies overlap the
 * solves.  An input buffer may appear more than once; an output buffer
 * written twice holds the later solve.  SF_ERR_ARG for a null table or
 * entry, n < 0; SF_ERR_STATE on a batch.  The paper has no counterpart (its
 * solver works on host memory one call at a time). */
sf_status sf_solve_host_many(sf_plan p, int n, const void *const *host_f, void *const *host_psi,
                             void *const *host_op_out);

/* Transposed solve for gradients: given dL/dpsi (g_psi, may be NULL) and
 * dL/d(op output) (g_op, may be NULL), write dL/df into g_f.  The solve is
 * affine in f; boundary data only shifts it, so it does not enter here.
 * Same pass structure as the solve with the multiplier applied to the
 * conjugate-transposed operator (the paper has no adjoint; this is the
 * exact transpose of the discrete map).  For first derivatives on Dirichlet /
 * Neumann axes the operator gradient is first mapped onto a psi gradient by
 * transposed derivative passes into plan-owned workspace. */
sf_status sf_solve_adjoint(sf_plan p, const void *dev_g_psi, const void *dev_g_op, void *dev_g_f);

/* Batched solve of independent problems in one CUDA graph (one persistent
 * kernel launch for the members on the general engine).
 * plans: n plans of the same precision (their own stream is ignored; the
 * batch uses cuda_stream).  The batch references the plans' tables and owns
 * a work list and workspace; destroy it before its plans. */
sf_status sf_batch_create(sf_plan *batch, const sf_plan *plans, int n, void *cuda_stream);

/* Enqueue one batched solve: f[i], psi[i], op[i] are the i-th problem's
 * buffers (op may be NULL, or op[i] NULL when that plan has no operator).
 * The first call captures the launch sequence into a CUDA graph that later
 * calls replay while the pointers stay the same.  Members on the register
 * fast path run their own three launches in that graph after the persistent
 * launch of the other members; their buffers are kernel arguments, so a
 * change of buffers re-captures the graph, and the first call also solves
 * those members once outside the graph. */
sf_status sf_batch_solve(sf_plan batch, const void *const *f, void *const *psi, void *const *op);

/* Wait for the plan's stream and report device-side status (SF_ERR_TIMEOUT if
 * a scheduler wait gave up, SF_ERR_CUDA on an asynchronous CUDA error,
 * SF_ERR_CORRUPT if a guard band of an SF_FLAG_DEBUG_CHECKS plan changed). */
sf_status sf_sync(sf_plan p);

/* Kernel launches one sf_execute / sf_batch_solve enqueues (for accounting). */
int sf_plan_launches(sf_plan p);

/* Tracing of the last persistent-executor launch of a plan (waits for the
 * plan's stream).  For each of up to 8 pass kinds k (register path: 0 = y
 * forward, 1 = z stage, 2 = y inverse; general engine: the pass kind of the
 * tile, kinds 8 to 11 -- the 1D multiply and the derivative passes -- counted
 * with kinds 0 to 3): out[3k] = summed tile time (ns, over all CTAs),
 * out[3k+1] = summed time spent waiting for dependencies (ns), out[3k+2] =
 * tiles.  out must hold 24 doubles.  The paper times the solve steps separately (Sec. 5.3); this is
 * the per-pass breakdown of the GPU schedule. */
sf_status sf_plan_stats(sf_plan p, double out[24]);

/* Per-kernel CUDA-event timing of a plan (diagnostic, off by default).
 * enable = 1 creates the events on first use and clears the record; from then
 * on every full solve (sf_solve, sf_execute, sf_solve_host) records an event on
 * the plan's stream before its first kernel, between consecutive kernels and
 * after its last one.  enable = 0 stops recording.  Waits for the plan's
 * stream.  Solves enqueued while the stream is being captured into a graph are
 * not recorded.  SF_ERR_ARG for a null plan or a batch. */
sf_status sf_plan_timing(sf_plan p, int enable);

/* Mean device time in milliseconds of each kernel slot over the solves
 * recorded since timing was enabled (the last 256 at most); waits for the
 * plan's stream.  Register fast path: 3 slots (ms[0] x forward transform,
 * ms[1] the y/z executor, ms[2] x inverse transform); general engine: 1 slot
 * (the executor, all its launches).  ms must hold 4 doubles; unused slots are
 * 0.  *nslot and *nsolve (either may be NULL) receive the slot count and the
 * number of solves averaged (0 when nothing was recorded). */
sf_status sf_plan_kernel_ms(sf_plan p, double ms[4], int *nslot, int *nsolve);

/* A bounded solve that allocates nothing, for callers that cannot call
 * cudaMalloc (code inside host callbacks or driver hooks that must not
 * allocate, real-time loops that forbid allocation after start-up, processes
 * whose device memory is owned by another allocator).  There is no
 * counterpart in the paper: it is the plan-based solve (sf_plan_create +
 * sf_execute) without a plan, restricted to what fits a fixed workspace.
 *   d        problem description; FP32, one component, no operator, periodic /
 *            Dirichlet / Neumann axes only (homogeneous boundaries), 2D or 3D.
 *   dev_f    device source, dev_psi device result (layouts as for sf_execute).
 * Workspace and tables live in one file-scope device array of 64 MiB that
 * every GPU loading this library holds until the process exits.  A problem
 * whose workspace does not fit returns SF_ERR_ARG (use sf_plan_create); other
 * unsupported options return SF_ERR_UNSUPPORTED; sf_last_error gives the
 * reason (for an oversized problem, the bytes it would need).  No cudaMalloc,
 * cudaFree or other allocation is made.  Set-up: the first call in each CUDA
 * context on a device (the first call on that device, and again the first
 * after a cudaDeviceReset or in another driver-API context) looks up the
 * array's device address (cudaGetSymbolAddress) and sets the kernel's shared
 * memory attribute; that call must come before any stream capture.  All calls
 * share the array and it keeps the last call's contents: calls that may
 * overlap on the GPU (other streams, other threads) race and corrupt each
 * other's results.  Work is enqueued on cuda_stream; the result is ready when
 * that stream reaches it. */
sf_status sf_solve_static(const sf_plan_desc *d, const void *dev_f, void *dev_psi, void *cuda_stream);

/* Self-test of the bounded waits of the persistent scheduler: launches a
 * two-pass work list whose second pass depends on a tile count the first pass
 * can never reach (a flag nothing sets), with the given wait limit in
 * milliseconds, on cuda_stream.  Every wait gives up after the limit, the
 * kernel exits normally and the status word is read back: the call returns
 * SF_ERR_TIMEOUT when the failure was detected as designed (SF_OK would mean
 * the wait did not give up).  No work is done on user data. */
sf_status sf_selftest_timeout(int timeout_ms, void *cuda_stream);

/* Test hooks for failure handling (the paper has no counterpart).
 * sf_debug_fail_alloc(after): every device allocation the library makes from
 *   now on fails with SF_ERR_OOM once `after` more allocations have succeeded
 *   (after < 0 turns the injection off).  Plan creation then returns SF_ERR_OOM
 *   and releases what it had allocated.  Process-wide; not thread-safe.
 * sf_debug_corrupt_guard(p): overwrites one byte of the first guard band of a
 *   plan created with SF_FLAG_DEBUG_CHECKS (a host-issued cudaMemset into the
 *   plan's own allocation, so no kernel writes out of range); the next sf_sync
 *   must report SF_ERR_CORRUPT.  SF_ERR_STATE for a plan without debug checks. */
sf_status sf_debug_fail_alloc(int after);
sf_status sf_debug_corrupt_guard(sf_plan p);

/* Measured FP32 FMA throughput of the current device in TFLOP/s (one FMA =
 * 2 flop): 8 independent FMA chains per thread on 8 CTAs x 256 threads per
 * SM, one launch of about 30 ms timed with CUDA events on cuda_stream (NULL:
 * the legacy default stream), after one shorter warm-up launch.  It is the
 * measured counterpart of the unit-count FP32 peak against which the
 * register fast path (bound by instruction issue and the shared-memory pipe,
 * not by DRAM) is quoted; the paper has no such step.  SF_ERR_ARG for a null result pointer, SF_ERR_CUDA on a CUDA error. */
sf_status sf_probe_fp32_fma(double *tflops, void *cuda_stream);

/* The FP64 special functions with which plan set-up tabulates the kernels,
 * evaluated on the host for n points x[i] -> out[i] (no GPU needed; the same
 * code runs on the GPU when a plan builds its Green's table).  The paper has
 * no such step; the call exists so that this code can be checked against
 * independent implementations.  which = 0: the sine integral Si(x), x >= 0;
 * 1: F(x) = int_0^x (1 - J0(t)) / t dt, x >= 0 (2D spectral kernel);
 * 2: the exponential integral E1(x), x > 0 (2D Gaussian kernels).
 * SF_ERR_ARG for null pointers, n < 0 or an unknown `which`. */
sf_status sf_eval_special(int which, int n, const double *x, double *out);

/* Release a plan or batch and its device memory (waits for its stream). */
sf_status sf_plan_destroy(sf_plan p);

const char *sf_status_string(sf_status s);
const char *sf_last_error(void);

/* Library version string. */
const char *sf_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SAILFISH_GB300_H */
