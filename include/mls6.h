/*
 * mls6.h -- C ABI of the GB300 (sm_103a) multilevel summation library for
 * r^-6 dispersion.
 *
 * Method: Tameling, Springer, Bientinesi, Ismail, "Multilevel Summation for
 * Dispersion: A Linear-Time Algorithm for r^-6 Potentials", arXiv 1308.4005.
 * The kernel 1/r^6 is split (Eq. complete-splitting) into a local part g_0
 * (cutoff a, evaluated as a cell-list pair sum) and grid parts g_1..g_l that
 * are anterpolated to the finest grid, restricted, evaluated per level
 * (cutoff stencil 2^k a on levels k < l, periodic all-to-all table on level
 * l), prolongated and interpolated back (Sec. II.B), minus the self term
 * gamma(0)/a^6 xi^T xi (Eq. self-interaction-energy).
 *
 * Conventions
 *   energy  E = -1/2 sum_i sum_{j,n}' c_i c_j |x_i - x_j + n L|^-6  (MLS
 *           approximation of it), i.e. the quadratic form of
 *           Eq. (pot-vec-mat-vec) with xi = c (geometric mixing,
 *           Eqs. xi-general / xi-lj-geometric, c_i = sqrt(C6_i)), halved for
 *           the double sum and with the attractive sign of Eq. (disp-pair-pot).
 *   forces  F_i = -dE/dx_i, the exact gradient of the MLS energy (the paper
 *           does not print a force formula).
 *   virial  W_ab = -dE/d eps_ab under the affine strain x -> (1+eps) x of
 *           atoms, box and grids; six doubles in the order xx yy zz xy xz yz.
 *   box     orthorhombic and periodic in all three directions (Sec. II.C:
 *           only periodic boundaries are treated).
 *   grids   level k (1..l) has n_k = n_1 / 2^(k-1) points per axis and
 *           spacing h_k = 2^(k-1) L/n_1; node mu sits at mu * h_k.  n_1 is,
 *           per axis, the multiple of 2^(l-1) nearest to L/h (ties to the
 *           finer grid) -- non-power-of-two grids are allowed (Sec. III.C).
 *   basis   the cubic Hermite Phi of Eq. (Phi-Hermite), interpolation order
 *           p = 3 (the only order implemented).
 *
 * Threading and streams: a plan is not thread-safe; calls on one plan must
 * be serialised by the caller.  Work is enqueued on the plan's stream (the
 * legacy default stream unless mls6_set_stream was called).
 * Errors are returned as negative mls6_status codes; nothing aborts and
 * there is no CPU fallback: without a usable CUDA device every call that
 * needs one returns MLS6_ERR_CUDA.
 */
#ifndef MLS6_H
#define MLS6_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mls6_plan_t mls6_plan_t;

typedef enum {
  MLS6_OK = 0,
  MLS6_ERR_ARG = -1,        /* NULL pointer, N < 0, a <= 0, h <= 0, bad level ... */
  MLS6_ERR_GRID = -2,       /* grid sizes not nested / too many levels */
  MLS6_ERR_BOX = -3,        /* non-positive or non-finite box */
  MLS6_ERR_ORDER = -4,      /* interpolation order other than 3 or 5 */
  MLS6_ERR_CUDA = -5,       /* a CUDA runtime call failed (no device, launch error) */
  MLS6_ERR_NOMEM = -6,      /* device allocation failed */
  MLS6_ERR_TIMEOUT = -7,    /* a bounded device-side wait ran out (kernel gave up) */
  MLS6_ERR_NONFINITE = -8,  /* a position or coefficient was NaN/Inf */
  MLS6_ERR_SIZE = -9        /* request larger than a fixed capacity */
} mls6_status;

typedef enum {
  MLS6_FP64 = 0,  /* every step in double precision */
  MLS6_FP32 = 1,  /* pair kernel and grids in float; coarsest level, energy
                     and virial accumulation in double */
  MLS6_MIXED = 2  /* as MLS6_FP32, but the level stencils run on the tensor
                     cores with BF16 hi+lo split operands and FP32
                     accumulation (relative error of a stencil product
                     <= 3 * 2^-18); used when every tap row spans at most 8
                     nodes either side (2a/h_1 < 9), else the FP32 stencil */
} mls6_precision;

/* Finest-grid size for a box (per axis the multiple of 2^(levels-1) nearest
 * to L/h, ties to the finer grid: every coarser level then halves the node
 * count, Sec. II.A.4, and the rule gives the 12 x 12 x 192 grid of the slab
 * example in Sec. III.C).  Host only; needs no GPU.
 * box: 3 doubles (Lx, Ly, Lz).  n_out: 3 ints.  Returns MLS6_OK or an error
 * (MLS6_ERR_SIZE for a finest grid of more than 2^31 - 1 nodes, which the
 * grid kernels cannot index; mls6_plan returns the same). */
int mls6_grid_dims(const double box[3], double h, int levels, int n_out[3]);

/* Coarsest-level periodic tables (Eqs. last-grid-periodic and
 * last-grid-periodic-transformed): T[m] = sum_{n in Z^3} g_l(|m h_l + n L|)
 * for the nl[0] x nl[1] x nl[2] offsets m (x fastest), and the virial tables
 * V[c * n_l + m] = sum_n g_l'(r)/r r_a r_b for the six components c.  The
 * lattice sums are evaluated by Ewald summation of r^-6.  Host only; needs
 * no GPU.  T: nl0*nl1*nl2 doubles, V: 6 times that (may be NULL). */
int mls6_coarse_tables(const double box[3], const int nl[3], int levels, double a, double* T,
                       double* V);

/* Create a plan: the set-up of the method's algorithmic steps (Sec. II.B)
 * for one box and one atom count.  Validates the parameters, computes the
 * nested grid hierarchy (Sec. II.A.4, spacing 2^(k-1) h on level k), the
 * level-stencil table g_1(|m h_1|) for |m h_1| < 2a (Eq. g_k; the same table
 * serves every level k < l, scaled by 2^(-6(k-1))), the coarsest-level
 * periodic table (Eq. last-grid-periodic-transformed, Ewald-summed) and the
 * self term gamma(0)/a^6 (Eq. self-interaction-energy), all on the host in
 * FP64, and allocates all device workspace (the plan owns it).
 *   box        3 doubles (Lx, Ly, Lz), host
 *   N          number of atoms (>= 0), fixed for the plan
 *   a          local cutoff (> 0), the split radius of Eq. (g_0)
 *   h          requested finest spacing (> 0); the actual spacing per axis
 *              is L/n_1 (mls6_grid_dims)
 *   levels     number of grid levels l (1..12), or 0 for the automatic rule
 *              of mls6_auto_levels
 *   order      interpolation order p of the nodal basis Phi (Eq. def-phi):
 *              3 = Eq. (Phi-Hermite), the cubic C^1 interpolant (4 nodes per
 *              axis); 5 = the C^1 quintic (6 nodes per axis) whose orders
 *              Sec. III.B compares: even, piecewise quintic, support
 *              |t| < 3, reproducing polynomials of degree <= 4, the member
 *              whose outer piece continues to a root at |t| = 4:
 *                |t|<=1: (1-t^2)(2-|t|)(6+3|t|-5t^2)/12
 *                1..2:   (|t|-1)(|t|-2)(|t|-3)(5t^2-9|t|-4)/24
 *                2..3:  -(|t|-1)(|t|-2)(|t|-3)^2(|t|-4)/24
 *              Order-5 plans run the chained launch form in a batch and are
 *              refused by the learned correction (features are defined on
 *              the cubic basis).  Other values return MLS6_ERR_ORDER.
 *   precision  an mls6_precision value, passed as a plain int (the ABI has
 *              no options struct; the stream is set with mls6_set_stream)
 *   *out       receives the plan (NULL on error)
 * Errors: MLS6_ERR_ARG / _BOX / _GRID / _ORDER for bad parameters,
 * MLS6_ERR_NOMEM / _CUDA for device failures; nothing is leaked. */
int mls6_plan(mls6_plan_t** out, const double box[3], int64_t N, double a, double h, int levels,
              int order, int precision);

/* Plan options beyond mls6_plan's arguments (zero-initialise for the
 * defaults).
 *   continuity  C^n smoothing function, n in 1..4; 0 means 2 (Eq. gamma).
 *               The paper builds gamma from the electrostatic smoothing
 *               functions (Sec. II.A.3) and compares C^1 .. C^4 (Sec. III.B)
 *               but prints only n = 2; with u = rho^12, rho^-6 = u^(-1/2) and
 *               gamma_n is its Taylor polynomial about u = 1 to order n
 *               (n = 2 reproduces Eq. gamma), rho^-6 for rho >= 1.  It
 *               changes g_0 .. g_l, the tables and the self term
 *               gamma_n(0)/a^6.  Plans with n != 2 run the per-atom pair
 *               kernel only (pair_split 1..8) and refuse mls6_eval_lb.
 *   stencil     level-stencil kernel of an MLS6_MIXED plan: 0 automatic
 *               (tcgen05 tensor cores when 2a/h_1 < 9 and the levels give
 *               at least two 16^3 tiles per SM of the device, else the FP32
 *               CUDA-core kernel), 1 the FP32 CUDA-core kernel, 2 tcgen05
 *               tensor cores whenever 2a/h_1 < 9.  Ignored in FP64 / FP32.
 * Out-of-range values return MLS6_ERR_ARG. */
typedef struct {
  int continuity;
  int stencil;
} mls6_plan_options;

/* As mls6_plan, with options (NULL = defaults). */
int mls6_plan_ex(mls6_plan_t** out, const double box[3], int64_t N, double a, double h,
                 int levels, int order, int precision, const mls6_plan_options* opts);

/* Enqueue subsequent work of the plan on a cudaStream_t (NULL = legacy
 * default stream).  Internally an evaluation runs on two streams owned by
 * the plan (the pair sum in parallel with the grid chain); they wait for
 * the caller's stream at the start and the caller's stream waits for them
 * at the end, so ordering is as if all work ran on the caller's stream. */
int mls6_set_stream(mls6_plan_t* p, void* stream);

/* Graph execution (default on): the first evaluation with a given set of
 * pointers and options captures the whole kernel sequence into a CUDA
 * graph, later evaluations with the same pointers replay it (re-captured
 * when pointers, virial or profiling change).  enable = 0 launches the
 * kernels one by one. */
int mls6_set_graph(mls6_plan_t* p, int enable);

/* Evaluate energy, forces and virial: one pass of the method's five steps
 * (Sec. II.B: anterpolation, restriction, evaluation on every level,
 * prolongation, interpolation) plus the local pair sum of Eq. (g_0), i.e.
 * the quadratic form of Eq. (pot-vec-mat-vec) with xi = c, split as in
 * Eq. (pot-initial-splitting).
 *   pos     N rows of the plan's precision (double or float): if c == NULL
 *           each row is {x, y, z, c} (4 values), otherwise {x, y, z}
 *           (3 values).  Positions may lie anywhere; they are wrapped into
 *           the box.  Read only, by the binning kernel alone: device memory,
 *           or page-locked host memory (cudaHostAlloc, cudaMallocHost,
 *           cudaHostRegister) that the kernel reads over the host link with
 *           no separate copy; other host memory returns MLS6_ERR_ARG.  With
 *           host memory the caller keeps it unchanged until the evaluation
 *           has finished on the plan's stream.
 *   c       N coefficients c_i = sqrt(C6_i) (plan precision), device or
 *           page-locked host memory as pos, or NULL (coefficients in the 4th
 *           column of pos).
 *   forces  device pointer, N x 3 of the plan precision, overwritten
 *           (page-locked host memory also works; other host memory returns
 *           MLS6_ERR_ARG).
 *   energy  one double, host or device pointer, or NULL to skip.
 *   virial  six doubles (xx yy zz xy xz yz), host or device, or NULL to skip
 *           (skipping it also skips the virial arithmetic).
 * The call is asynchronous on the plan's stream unless energy or virial is a
 * host pointer, in which case it returns after the stream has finished.
 * NaN/Inf inputs are detected on the device; the status is reported by the
 * call when it synchronises, else by mls6_last_error.  N = 0 gives E = 0. */
int mls6_eval(mls6_plan_t* p, const void* pos, const void* c, void* forces, double* energy,
              double* virial);

/* As mls6_eval, and also writes the per-atom energies
 * -1/2 c_i (e0_i + e_i) + 1/2 (gamma(0)/a^6) c_i^2 (they sum to E; the
 * terms of Eq. pot-initial-splitting taken atom by atom, the last one the
 * self term of Eq. self-interaction-energy) to the device array atom_energy
 * (N doubles; other host memory than page-locked returns MLS6_ERR_ARG). */
int mls6_eval_atoms(mls6_plan_t* p, const void* pos, const void* c, void* forces, double* energy,
                    double* virial, double* atom_energy);

/* Lorentz-Berthelot mixing (Sec. II.D): sigma_ij = (sigma_i + sigma_j)/2,
 * eps_ij = sqrt(eps_i eps_j), pair coefficient C_ij = 2 eps_ij sigma_ij^6, so
 * E = -1/2 sum_i sum_{j,n}' C_ij |x_i - x_j + nL|^-6 (MLS approximation).
 * The local part uses C_ij exactly; the grid part runs once per channel of
 * the binomial expansion C_ij = sum_k xi_{i,k} xi_{j,6-k},
 * xi_{i,k} = (1/8) sigma_i^k sqrt(binom(6,k) 2 eps_i) (Eq.
 * disp-pair-pot-multilevel-LorentzBerthelot, seven instances of the
 * method), and the interpolation pairs channel k with 6-k.
 *   pos      N x 3 (plan precision), any positions
 *   sigma    N (plan precision), > 0
 *   epsilon  N (plan precision), >= 0
 *            (these three: device or page-locked host memory, as for
 *            mls6_eval's pos; other host memory returns MLS6_ERR_ARG)
 *   forces   device, N x 3, overwritten (as mls6_eval: MLS6_ERR_ARG for
 *            host memory that is not page-locked)
 *   energy   host or device double, or NULL
 * No virial.  Kernels are launched one by one (no graph) on the plan's
 * stream; a host energy makes the call wait and report MLS6_ERR_NONFINITE.
 * With all sigma_i equal the result equals mls6_eval with
 * c_i = sqrt(2 eps_i) sigma_i^3 (geometric mixing). */
int mls6_eval_lb(mls6_plan_t* p, const void* pos, const void* sigma, const void* epsilon,
                 void* forces, double* energy);

/* Waits for the plan's stream and returns the first device-detected error of
 * the last evaluation (MLS6_ERR_NONFINITE) or a pending CUDA error. */
int mls6_last_error(mls6_plan_t* p);

/* Plan geometry.  n_grid: 3*levels ints (points per axis, per level), may
 * be NULL; h_actual: 3 doubles (finest spacing), may be NULL; levels: may be
 * NULL; ntaps: number of stencil taps per level k < l, may be NULL. */
int mls6_plan_info(const mls6_plan_t* p, int* n_grid, double* h_actual, int* levels, int* ntaps);

/* Copy one grid of the last evaluation to host memory as doubles (x fastest):
 * which = 0: xi^k (anterpolated / restricted coefficients),
 *         1: e^k (level evaluation), 2: e^{k,tot} (after prolongation).
 * level: 1..l.  Synchronises the plan's stream. */
int mls6_debug_grid(mls6_plan_t* p, int level, int which, double* host_out);

/* Per-stage timing with CUDA events (off by default).  While enabled, the
 * evaluation runs its stages one after another on one stream (the pair
 * sum no longer overlaps the grid chain) and records an event at the start
 * and end of each stage:
 * 0 bin (wrap, cell histogram, scan, scatter, per-cell order), 1 pair
 * (local part), 2 anterpolation, 3 restriction, 4 level stencils,
 * 5 coarsest level, 6 prolongation, 7 interpolation/forces, 8 reduction. */
int mls6_profile(mls6_plan_t* p, int enable);

/* Waits for the plan's stream and writes the stage durations of the last
 * profiled evaluation (milliseconds) to ms[0..min(cap, stages)-1]; returns
 * the number of stages (>= 0) or an error.  *launches (may be NULL)
 * receives the number of kernels the last evaluation launched. */
int mls6_stage_times(mls6_plan_t* p, double* ms, int cap, int* launches);

/* Name of stage i (see mls6_profile), or NULL. */
const char* mls6_stage_name(int i);

/* Level count used when mls6_plan is given levels = 0: the largest l (1..12)
 * for which every axis of the coarsest grid of the hierarchy that
 * mls6_grid_dims(box, h, l) gives has at least 4 points (1 if already l = 2
 * fails).  The paper leaves l to the user (Sec. II.A.4: any number of
 * nested grids; Sec. IV: the coarsest product costs N_l^2 and must stay
 * small); this rule keeps N_l at 64..~500 nodes.  Host only; returns l >= 1
 * or a negative status. */
int mls6_auto_levels(const double box[3], double h);

/* Kernel shapes of a plan.  pair_split selects the local pair kernel:
 * 1, 2, 4 or 8 lanes per atom (each lane group walks its atom's neighbour
 * cells); 16, 32: warp form (two or one atoms per warp share one flattened,
 * row-trimmed candidate stream, every candidate evaluated branch-free);
 * 128, 256, 512: queue form (2, 4 or 8 atoms per warp share that stream,
 * staged in shared memory; the lanes test 32 candidates at a time and the
 * pairs inside the cutoff are queued and evaluated 32 at a time on full
 * warps); 1024: cluster form (FP32 and mixed plans: a warp pairs 8
 * consecutive sorted atoms with every candidate of their segment's
 * neighbour cells, four candidates per step, branch-free; Lorentz-Berthelot
 * evaluations of such a plan run the one-lane-per-atom kernel).  The warp
 * and queue forms are refused with MLS6_ERR_ARG when the neighbour range
 * spans more than two cells per side or the box has fewer than five cells
 * along x, the cluster form also in FP64 or with fewer than 16 cells along
 * x.  stencil_groups: thread groups of 128 sharing one 8^3 stencil tile (1,
 * 2 or 4; ignored when the stencil tile does not fit in shared memory); 0
 * keeps the current value.  Defaults: FP64 the queue form with two atoms per
 * warp where allowed; otherwise the lanes per atom that give about 48
 * resident warps per SM (the cluster form is selected only by this call);
 * stencil: 24 warps per SM.  A shape
 * changes the order of floating-point sums (results move at rounding level),
 * never what is summed.  Waits for the plan's streams; the next evaluation
 * re-captures its graph. */
int mls6_set_tuning(mls6_plan_t* p, int pair_split, int stencil_groups);

/* Which level-stencil kernel the plan runs: 0 shared-memory tiles on the
 * CUDA cores (FP64 / FP32, and MLS6_MIXED plans whose grids are too small
 * for the tensor-core tiles), 1 global-memory fallback (tile and taps
 * beyond the shared-memory budget), 2 tensor cores through mma.sync
 * (MLS6_MIXED, not chosen while 3 applies), 3 tensor cores through tcgen05
 * with the accumulators in tensor memory (MLS6_MIXED, 2a/h_1 < 9, see
 * mls6_plan_options), -1 none (l = 1). */
int mls6_stencil_kind(const mls6_plan_t* p);
int mls6_get_tuning(const mls6_plan_t* p, int* pair_split, int* stencil_groups);

/* ---------------------------------------------------------------------
 * Batches: B independent replicas (each its own box, atom count and grid
 * hierarchy, same a, h, levels rule, order and precision) evaluated by a
 * single CUDA graph launch.  FP32 batches can run one persistent kernel
 * instead (see mls6_batch_set_mode); by default the replicas' kernel sequences are
 * captured into K independent chains of the graph (branches), replicas
 * assigned to chains by longest-processing-time-first on the cost model
 * below.  Each replica runs the kernels (or kernel bodies) of a single plan
 * with the same shapes, so its results equal mls6_eval's on such a plan bit
 * for bit.
 * --------------------------------------------------------------------- */
typedef struct mls6_batch_t mls6_batch_t;

/* Model run time (seconds) of one evaluation, after the paper's cost
 * model (Sec. IV, Eq. cost: C_local (a/d)^3 N + C_grids (a/h)^3 V/h^3 with
 * d^3 = V/N) extended by a per-atom term (binning, anterpolation,
 * interpolation), the coarsest product N_l^2 and a per-launch latency:
 *   coef[0] (a^3 N/V) N + coef[1] (a/h)^3 (V/h^3) 8/7 + coef[2] N
 *   + coef[3] N_l^2 + coef[4] (8 + 2(l-1)).
 * coef: 5 doubles or NULL for the built-in values (from GB300 stage
 * timings).  Host only. */
int mls6_cost_model(const double box[3], int64_t N, double a, double h, int levels,
                    const double* coef, double* cost);

/* Longest-processing-time-first assignment of B jobs of the given costs to
 * K chains: jobs in decreasing cost (stable), each to the chain with the
 * least load so far (lowest index on ties).  branch_of: B ints, written;
 * load: K doubles (may be NULL), written.  Host only. */
int mls6_lpt_assign(int B, const double* cost, int K, int* branch_of, double* load);

/* Create a batch.  boxes: B x 3 doubles; N: B atom counts; a, h, levels
 * (0 = mls6_auto_levels per replica), order, precision as for mls6_plan.
 * The batch owns the B plans and a few per-replica words.  On error no
 * batch is returned and everything allocated is released. */
int mls6_batch_plan(mls6_batch_t** out, int B, const double* boxes, const int64_t* N, double a,
                    double h, int levels, int order, int precision);

/* Stream ordering as for mls6_set_stream. */
int mls6_batch_set_stream(mls6_batch_t* b, void* stream);

/* Evaluate all replicas.  pos, c, forces: device arrays concatenating the
 * replicas in order (replica r starts at atom offsets[r] of
 * mls6_batch_size), laid out as for mls6_eval (page-locked host memory also
 * works; other host memory returns MLS6_ERR_ARG, here and in
 * mls6_batch_tune).  energy: B doubles, virial:
 * 6B doubles (NULL skips the virial), host or device; host pointers make the
 * call wait and report MLS6_ERR_NONFINITE if any replica saw a non-finite
 * input.  The first call with a set of pointers captures the graph. */
int mls6_batch_eval(mls6_batch_t* b, const void* pos, const void* c, void* forces,
                    double* energy, double* virial);

/* Autotune on the given inputs: times whole-batch launches (median of reps,
 * with the virial) while it varies the branch count over 1..64, then the
 * lanes per atom and the stencil groups of every replica one power of two
 * below and above their defaults, keeping each change that lowers the time.
 * For FP32 batches that the persistent kernel can run, the other launch
 * form (mls6_batch_set_mode) is tuned as well and the faster form is kept.
 * Leaves the best configuration applied; best_sec (may be NULL) receives
 * its time.  forces is overwritten. */
int mls6_batch_tune(mls6_batch_t* b, const void* pos, const void* c, void* forces, int reps,
                    double* best_sec);

/* Set the configuration directly: branches (0 keeps it; chains are
 * re-assigned by LPT), per-replica pair_split / stencil_groups arrays of B
 * ints (NULL keeps them; 0 entries keep that replica's value). */
int mls6_batch_set_config(mls6_batch_t* b, int branches, const int* pair_split,
                          const int* stencil_groups);

/* Current configuration; each array of B ints/doubles may be NULL:
 * branch count, per replica lanes per atom, stencil groups, chain index,
 * model cost (seconds) and level count; launches: kernels in the graph
 * captured last (0 before the first evaluation). */
int mls6_batch_info(const mls6_batch_t* b, int* branches, int* pair_split, int* stencil_groups,
                    int* branch_of, double* cost, int* levels, int* launches);

/* The plan of replica r, owned by the batch (valid until the batch is
 * destroyed): for mls6_plan_info, mls6_profile / mls6_stage_times on a
 * single evaluation of that replica, or mls6_debug_grid.  Changing its
 * shapes with mls6_set_tuning directly bypasses the batch's graph: use
 * mls6_batch_set_config instead. */
int mls6_batch_replica(mls6_batch_t* b, int r, mls6_plan_t** plan);

/* Number of replicas and the B+1 atom offsets (may be NULL). */
int mls6_batch_size(const mls6_batch_t* b, int* B, int64_t* offsets);

/* Execution mode.  persistent = 1: when every replica is FP32
 * with at least two levels, the shared-memory stencil kernel and 1..8 pair
 * lanes per atom, the graph holds one persistent kernel: its blocks take
 * (stage, replica, block) work items from a device queue in stage-major
 * order (replicas in decreasing cost within a stage), wait until the
 * replica's previous stage has counted all its blocks (bounded waits, see
 * mls6_batch_set_wait), run the same kernel body as the per-stage launch,
 * and count the item done.  Results equal mls6_eval's on each replica's
 * plan bit for bit.  persistent = 0 (default), or an ineligible batch: the
 * graph of per-replica kernel chains described above.  Waits for the
 * batch's work; the next evaluation re-captures. */
int mls6_batch_set_mode(mls6_batch_t* b, int persistent);

/* 1 if the batch's graph runs (or, before its next capture, will run) the
 * persistent kernel, 0 otherwise. */
int mls6_batch_mode(const mls6_batch_t* b);

/* Bounded waits of the persistent kernel: a block polls a replica's stage
 * counter at most `limit` times (about 0.1 us apart; default 2^22, i.e. well
 * under a second) before it records a timeout and every block leaves the
 * kernel; the call then reports MLS6_ERR_TIMEOUT (host energy pointers, or
 * mls6_batch_last_error).  withhold >= 0 is a test hook: the item with that
 * number never counts as done, so the waits behind it run out (no fault, no
 * trap: the kernel returns).  -1 disables it.  Takes effect at the next
 * evaluation. */
int mls6_batch_set_wait(mls6_batch_t* b, long long limit, long long withhold);

/* Waits for the batch's work and returns MLS6_ERR_TIMEOUT if the persistent
 * kernel's bounded wait ran out, MLS6_ERR_NONFINITE if a replica saw a
 * non-finite input, else MLS6_OK. */
int mls6_batch_last_error(mls6_batch_t* b);

/* Release the batch, its plans and all their device memory.  NULL is ignored. */
void mls6_batch_destroy(mls6_batch_t* b);

/* ---------------------------------------------------------------------
 * Learned force correction for a coarse grid.  The paper has no
 * counterpart: a small network reads each atom's neighbourhood of the
 * level-1 total potential e^{1,tot} of a (coarse) evaluation and predicts
 * the force residual to a finer evaluation; forces += c_i * s * y_i.  The
 * plain evaluation is unchanged and remains the reference.
 *
 * Features (per atom, input order, 128 per row): for the 27 offsets d in
 * {-1,0,1}^3 (x fastest) the potential and its gradient (4 values)
 * interpolated with the method's basis (Eq. interpolation) at x_i + h_1 d,
 * then sin and cos of 2 pi times the fractional level-1 grid coordinate of
 * x_i per axis, zero padding; each normalised as (f - shift_j) * scale_j.
 * Network: 128 -> 64 -> 64 -> 64 -> 8 (outputs 0..2 used), tanh hidden
 * layers, BF16 weights and activations on the tensor cores with FP32
 * accumulation.  Parameters: one FP32 vector of mls6_mlp_n_params() values,
 * W1 (128 x 64, row = input) b1 W2 (64 x 64) b2 W3 b3 W4 (64 x 8) b4.
 * Training: loss (1/N) sum_i sum_{c<3} (y_ic - t_ic)^2; the backward pass
 * runs on the tensor cores in BF16 with FP32 accumulation (activation
 * gradients dZ = (dZ' W^T)(1 - h^2) kept in BF16, weight gradients X^T dZ
 * and H^T dZ, bias gradients as products with a ones operand), partial sums
 * over blocks of atoms reduced in a fixed order (reproducible bit for bit);
 * Adam (0.9, 0.999, 1e-8) on FP32 master weights.
 * Arrays described as device may also be page-locked host memory; other
 * host memory returns MLS6_ERR_ARG.
 * All calls are asynchronous on the model's stream (mls6_mlp_set_stream)
 * except where a host result is returned; calls that take a plan run on the
 * plan's stream.
 * --------------------------------------------------------------------- */
typedef struct mls6_mlp_t mls6_mlp_t;

int mls6_mlp_n_params(void);

/* New model: Glorot-uniform weights drawn from SplitMix64(seed), zero
 * biases, identity normalisation, output scale 1. */
int mls6_mlp_create(mls6_mlp_t** out, uint64_t seed);
int mls6_mlp_set_stream(mls6_mlp_t* m, void* stream);

/* Parameters to / from host memory (n must equal mls6_mlp_n_params());
 * setting them resets the optimiser state. */
int mls6_mlp_get_params(const mls6_mlp_t* m, float* host, int n);
int mls6_mlp_set_params(mls6_mlp_t* m, const float* host, int n);

/* Feature normalisation (host arrays of 128) and output scale s. */
int mls6_mlp_set_norm(mls6_mlp_t* m, const float* shift, const float* scale, float out_scale);

/* Normalised features of the plan's last evaluation, written to the device
 * array out (N x 128, fmt 0 = bf16, 1 = float), input order. */
int mls6_mlp_features(mls6_plan_t* p, const mls6_mlp_t* m, void* out, int fmt);

/* Network outputs Y (device, N x 8 floats) for features X (device, N x 128
 * bf16). */
int mls6_mlp_forward(mls6_mlp_t* m, const void* X, int64_t N, float* Y);

/* Gradient of the loss for targets T (device, N x 3 floats) into grad
 * (device, n_params floats; may be NULL) and the loss (host, may be NULL:
 * a host loss makes the call wait).  X (N x 128 bf16) must be 16-byte
 * aligned (its rows are copied in 16-byte pieces); MLS6_ERR_ARG otherwise. */
int mls6_mlp_grad(mls6_mlp_t* m, const void* X, const float* T, int64_t N, float* grad,
                  double* loss);

/* One Adam step on the batch (X, T) with learning rate lr (X aligned as
 * for mls6_mlp_grad). */
int mls6_mlp_train_step(mls6_mlp_t* m, const void* X, const float* T, int64_t N, float lr,
                        double* loss);

/* Correct the forces of the plan's last evaluation in place (device, N x 3
 * of the plan precision, input order): features, network, then
 * F_i += c_i * s * y_i.  Three kernels on the plan's stream. */
int mls6_mlp_apply(mls6_plan_t* p, mls6_mlp_t* m, void* forces);

void mls6_mlp_destroy(mls6_mlp_t* m);

/* Coarsest-level product that allocates no device memory.  The paper has no
 * counterpart: this is a library convenience for callers that may not
 * allocate device memory when they call in -- an MD engine that reserves
 * its whole memory budget up front, code where cudaMalloc/cudaFree would
 * synchronise the device or is not permitted, or a host framework whose
 * own allocator must not be bypassed.
 *   q       device, n[0]*n[1]*n[2] doubles: xi^l on the coarsest grid (x fastest)
 *   n       host, 3 ints: coarsest grid size; at most 4096 nodes in total,
 *           larger grids return MLS6_ERR_SIZE
 *   T, V    device: the tables of mls6_coarse_tables (V may be NULL when
 *           virial is NULL)
 *   e       device, n0*n1*n2 doubles, written: e_mu = sum_nu T[(mu-nu) mod n] q_nu
 *   virial  device, 6 doubles, written (or NULL):
 *           1/2 sum_mu q_mu sum_nu V_c[(mu-nu) mod n] q_nu
 *   stream  cudaStream_t (NULL = legacy default stream); asynchronous.
 * q, T, V, e and virial may also be page-locked host memory; other host
 * memory returns MLS6_ERR_ARG (checked after the grid size).
 * Its scratch (six doubles per node) is one fixed file-scope device array of
 * 192 KiB that every GPU loading the library holds until the process exits.
 * Every call looks up that array's device address in the current context
 * (cudaGetSymbolAddress), so a cudaDeviceReset leaves nothing stale.  The
 * first call on a device may load the library's kernels, so make it before
 * any stream capture.
 * All calls share the array and every entry a call reads is written by the
 * same call, so nothing needs clearing, but calls that overlap on the GPU
 * (different streams, or different host threads) race on it. */
int mls6_coarse_apply_noalloc(const double* q, const int n[3], const double* T, const double* V,
                              double* e, double* virial, void* stream);

/* Measured fused multiply-add rate of the current device (TFLOP/s, 2 flop
 * per FMA): precision MLS6_FP32 or MLS6_FP64.  A measurement tool for the
 * arithmetic rooflines of the pair and level-stencil kernels (the paper has
 * no counterpart): every SM runs independent FMA chains for ~20 ms, best of
 * five timed launches on the legacy default stream.  Synchronous; allocates
 * and frees a small device buffer. */
int mls6_fma_peak(int precision, double* tflops);

/* Release the plan and all its device memory.  NULL is ignored. */
void mls6_destroy(mls6_plan_t* p);

/* Static description of a status code. */
const char* mls6_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* MLS6_H */
