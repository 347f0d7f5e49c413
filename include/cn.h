/*
 * cn.h -- C ABI of the GB300-native fixed-step cable-network engine.
 *
 * The engine advances many multi-compartment cells with the fixed-step
 * (backward Euler) method of CoreNEURON (arXiv 1901.10975, Section 2): every
 * step delivers due events, assembles each cell's tree matrix from the
 * mechanism currents and conductances (Eq. 1), solves it by Gaussian
 * elimination in Hines order, updates the gating states and detects
 * threshold crossings; spikes are exchanged once per minimum-delay interval
 * (Section 2, hybrid clock-event algorithm).  All of that runs in CUDA
 * kernels for sm_103a; this header only carries plain pointers and sizes.
 *
 * Conventions shared by every entry point:
 *  - Each call returns a cn_status.  No exception crosses the ABI.  After a
 *    failure cn_last_error() describes it.
 *  - Host input arrays are copied; the caller keeps ownership and may free
 *    them when the call returns.  Outputs are written into caller buffers.
 *  - A model handle is not thread-safe: one host thread at a time.
 *  - Units: mV, ms, um, um2, uF/cm2, MOhm, S/cm2 (density mechanisms),
 *    uS (synaptic weights and conductances), nA (stimuli).
 *  - Indices are 0-based.  Node indices are global (concatenated cells, cell
 *    c owning nodes [cell_offset[c], cell_offset[c+1])) unless a field says
 *    "cell-local".
 */
#ifndef CN_H_
#define CN_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CN_OK = 0,
  CN_EINVAL = 1,    /* bad argument or inconsistent model description */
  CN_ENOMEM = 2,    /* device or host allocation failed */
  CN_ECUDA = 3,     /* a CUDA runtime call or kernel launch failed */
  CN_ESTATE = 4,    /* call not allowed in the model's current state */
  CN_ETIMEOUT = 5,  /* a bounded device wait gave up */
  CN_ERANGE = 6     /* a fixed-capacity buffer overflowed (see cn_last_error) */
} cn_status;

/* Mechanism types and their parameter columns (SoA, one column per name, in
 * this order).  Density mechanisms use S/cm2 and mV; point processes uS.
 * Gate kinetics of the channel types: alpha = A (v-vh)/(1-exp(-(v-vh)/k)),
 * beta = B exp(-(v-vh2)/k2), cnexp update (Section 6: fixed step).        */
typedef enum {
  CN_MECH_PAS = 0,    /* g, e                                                   */
  CN_MECH_HH = 1,     /* gnabar, gkbar, gl, el, ena, ek (Hodgkin-Huxley, 6.3 C)  */
  CN_MECH_EXPSYN = 2, /* tau, e   (point process; state g in uS)                 */
  CN_MECH_NA3H = 3,   /* gbar, erev, m:{A,vh,k,B,vh2,k2}, h:{...}   g = gbar m^3 h */
  CN_MECH_KDR4 = 4,   /* gbar, erev, n:{6}                          g = gbar n^4   */
  CN_MECH_KA = 5,     /* gbar, erev, a:{6}, b:{6}                   g = gbar a^3 b */
  CN_MECH_IH = 6,     /* gbar, erev, q:{6}                          g = gbar q     */
  CN_MECH_CAHVA = 7,  /* gbar, erev, m:{6}, h:{6}, depth, taur, cainf  g = gbar m^2 h,
                         cai' = -1e4 ica/(2 F depth) (inward) + (cainf-cai)/taur  */
  CN_MECH_KCA = 8,    /* gbar, erev, A, kd, B:  alpha = A cai/(cai+kd), beta = B */
  CN_MECH_NTYPES = 9
} cn_mech_type;

/* Number of parameter columns of a mechanism type (-1 for an unknown type). */
int32_t cn_mech_nparams(int32_t type);

typedef enum {
  CN_PREC_FP64 = 0,      /* everything FP64                                     */
  CN_PREC_GATE_FP32 = 1, /* gating rates, exponentials and state updates FP32   */
  CN_PREC_GATE_BF16 = 2  /* as GATE_FP32, gating states stored as bfloat16      */
} cn_precision;

/* Morphology (Section 2: a tree of compartments per cell, indexed by parent).
 * parent is cell-local with parent[i] < i and exactly one root (-1) per cell,
 * at cell-local index 0.  area and ri are per node; ri is the axial
 * resistance between a node and its parent (ignored at roots).            */
typedef struct {
  int32_t n_cells;
  const int32_t* cell_offset;   /* [n_cells+1], cell_offset[0] = 0 */
  const int32_t* parent;        /* [n_nodes], cell-local */
  const double* area_um2;       /* [n_nodes] */
  const double* cm_uF_cm2;      /* [n_nodes] */
  const double* ri_MOhm;        /* [n_nodes] */
  const int32_t* spike_node;    /* [n_cells], cell-local threshold-detection node */
  const double* threshold_mV;   /* [n_cells] */
} cn_morph;

/* One SoA mechanism instance table (Section 4.2: instances of one type are
 * grouped, each property stored contiguously).  param is [n_params][n]. */
typedef struct {
  int32_t type;
  int32_t n;
  const int32_t* node;          /* [n] global node index per instance */
  const double* param;          /* [cn_mech_nparams(type) * n] */
} cn_mech_table;

/* Device allocator used for every buffer of a model.  NULL -> cudaMalloc. */
typedef void* (*cn_alloc_fn)(size_t bytes, void* ctx);
typedef void (*cn_free_fn)(void* ptr, void* ctx);

typedef struct {
  double dt_ms;          /* time step (0.025 typical) */
  double v_init_mV;      /* initial voltage of every node; gates start at steady state */
  int32_t precision;     /* cn_precision */
  int32_t device;        /* CUDA device ordinal */
  void* stream;          /* cudaStream_t for every launch and copy (NULL: legacy default) */
  cn_alloc_fn alloc;
  cn_free_fn free;
  void* alloc_ctx;
  int32_t mapping;       /* CN_MAP_AUTO, CN_MAP_THREAD, CN_MAP_TUNE, or a target span (>= 16 rows) */
  int32_t use_graph;     /* nonzero: whole intervals replay, 8 at a time, from a captured CUDA graph */
  int32_t warps_per_block; /* 1..4 warps (each one group of 32 lanes) per block of the interval
                              kernel; 0 = 1 (CN_MAP_TUNE picks it) */
} cn_options;

/* Cell-to-lane mapping.  Cells are packed 32 lanes to a warp with
 * interleaved rows; a cell larger than the target span is cut into subtrees
 * ("parts") that occupy lanes of one warp and hand their junction values to
 * each other through a per-warp shared-memory mailbox (the warp-cooperative
 * solve of large cells); parts of several cells may stack in one lane.  A
 * value >= 16 sets the target span in rows directly.                      */
typedef enum {
  CN_MAP_TALL = 1 << 20, /* flag on a target span: every warp as tall as the largest cell span, so
                            that more parts stack in a lane (default: a warp is as tall as the
                            span of the cell that opened it) */
  CN_MAP_TALL2 = 1 << 21, /* flag on a target span: every warp twice the largest cell span
                             (with CN_MAP_TALL as well: 1.5 times the largest span) */
  CN_MAP_AUTO = 0,       /* target span = mean cell size (no split when the adjoint is on) */
  CN_MAP_THREAD = 1,     /* one cell per lane, never split */
  CN_MAP_INTERLEAVED = 3, /* reference layout, the paper's interleaved node ordering (Section 4.4):
                             one cell per lane, node i of every cell of a warp at row i; runs the
                             plain sequential form of each step (the linearised update of
                             Section 2 with no fused multiply-adds, IEEE divisions, every sum in
                             the order a per-cell stepper takes) so that results match such a
                             stepper up to its exp()'s last bit.  FP64 models of pas, HH,
                             ExpSyn and IClamp only (no channel types, gap junctions or
                             adjoint: CN_EINVAL) */
  CN_MAP_CONSTDEPTH = 4, /* reference layout, the paper's constant-depth node ordering (Section
                             4.4): a warp's 32 cells' nodes level by level (distance from the
                             root), one node per lane and row, never two children of one node in
                             one row; same arithmetic and limits as CN_MAP_INTERLEAVED */
  CN_MAP_TUNE = 2        /* autotuned on first use: each candidate layout (one cell per lane; spans
                            of 1/8, 1/4, 1/2 and 1 mean cell size, each also with CN_MAP_TALL,
                            CN_MAP_TALL | CN_MAP_TALL2 and CN_MAP_TALL2; then 0.85, 0.9, 0.95
                            and 1.1 times the best span; then, when the best has CN_MAP_TALL
                            alone, warp heights (CN_MAP_HEIGHT) at the best span and 3/4 of
                            it: the lowest height whose warps all fit on the device at once,
                            and that height + 4 rows)
                            with 1, 2 and 4 warps per block runs one timed interval from the
                            initial state; the fastest is kept */
} cn_mapping;

/* Warp height field of a mapping value (bits 22-30), with CN_MAP_TALL and a
 * target span: every warp is h rows tall (16 <= h <= 511) instead of the
 * largest cell span.  Cells whose span exceeds h are cut again with finer
 * targets (down to 4 rows per part) and open warps of their own span if
 * they still exceed it.  Parts then also fill the free runs of rows that a
 * part root's junction constraint leaves below a lane's top, and a part
 * goes where 4 x (padding rows left below it) + (rows of delay past its
 * earliest row) is least, else at the earliest row that fits.  Cells are
 * packed in up to 16 chunks of at least 1,024 cells each, on host threads;
 * the chunks follow from the cell count alone, so the layout does not
 * depend on the host.                                                     */
#define CN_MAP_HEIGHT_SHIFT 22
#define CN_MAP_HEIGHT_MASK ((int32_t)0x1ff << CN_MAP_HEIGHT_SHIFT)
#define CN_MAP_HEIGHT(h) ((int32_t)(h) << CN_MAP_HEIGHT_SHIFT)

/* The layout in use (after the first cn_run, or after the autotuner):
 * mapping (CN_MAP_THREAD or the target span), warps per block, warps in all,
 * and the autotuner's timed interval in ms (0 without tuning).  Lays the
 * model out first if needed.                                             */
typedef struct cn_model cn_model;
cn_status cn_get_mapping(cn_model* m, int32_t* mapping, int32_t* warps_per_block, int32_t* n_warps,
                         float* tuned_interval_ms);

/* Host-only preview of the placement cn_model_create makes for a morphology
 * (no GPU is touched), with the stacking of several cells' parts per lane
 * allowed.  The elimination order is the Hines order of Section 2: in every
 * part the rows are a depth-first preorder of its subtree, so a row's parent
 * is an earlier (lower) row of the same lane, or, for a part root, the
 * junction row of the parent part, at a lower warp row in any lane of the
 * same warp, reached through a per-warp mailbox entry.
 *   n_cells, cell_offset[n_cells+1], parent[n_nodes]: as in cn_morph.
 *   mapping: a cn_mapping value or a target span (>= 16 rows), optionally
 *   with CN_MAP_TALL, CN_MAP_TALL2 or both, or CN_MAP_TALL with a warp
 *   height CN_MAP_HEIGHT(h).
 * Outputs (caller-owned, each may be NULL):
 *   node_lane[n_nodes]  global lane = 32 * warp + lane of the node's part
 *   node_row[n_nodes]   warp row of the node
 *   node_flags[n_nodes] topology bits: 1<<6 the in-part parent is not the
 *                       previous row ("far"); bits 7-9 number of far
 *                       children; 1<<11 real node; 1<<12 junction (a child
 *                       part hangs from it) with the mailbox entry in bits
 *                       14-22; 1<<13 part root with its mailbox entry in
 *                       bits 23-31 (bits 0-5 and 10 are filled at model
 *                       creation: mechanism slot, pas).
 *   n_warps, stack_depth: warps used; the most far children pending at
 *                       once in any lane while it is eliminated (a bound on
 *                       the entries of the kernel's per-lane stack).
 * With CN_MAP_INTERLEAVED or CN_MAP_CONSTDEPTH the reference placement is
 * returned (spike sources taken at each cell's root; node_flags then only
 * marks real nodes).
 * Errors: CN_EINVAL on malformed trees or a node with more than 8 children. */
cn_status cn_plan_layout(int32_t n_cells, const int32_t* cell_offset, const int32_t* parent, int32_t mapping,
                         int32_t* node_lane, int32_t* node_row, int32_t* node_flags, int32_t* n_warps,
                         int32_t* stack_depth);

/* Fill *opt with defaults: dt 0.025 ms, v_init -65 mV, FP64, device 0,
 * default stream, cudaMalloc, autotuned mapping, graphs on. */
void cn_options_default(cn_options* opt);

/* Geometry helper (Section 2 discretisation, the engine's reading): each node
 * is a cylinder of length dx and diameter diam; area = pi diam dx (lateral
 * surface); the half-segment resistance is 1e-2 * 2 Ra dx / (pi diam^2) MOhm
 * and ri(node) = R_half(node) + R_half(parent).  parent is cell-local as in
 * cn_morph.  Outputs area[n_nodes] and ri[n_nodes] (0 at roots).
 * Errors: CN_EINVAL on bad parent indices or non-positive geometry.      */
cn_status cn_geometry(int32_t n_cells, const int32_t* cell_offset, const int32_t* parent,
                      const double* dx_um, const double* diam_um, const double* Ra_ohm_cm,
                      double* area_um2, double* ri_MOhm);

/* Build a model on the GPU from a morphology and mechanism tables (Eq. 1's
 * terms: pas -> I_pas, channels -> I_ion, EXPSYN -> I_syn; Section 4.2 SoA
 * tables).  At most one table per type.  Every node must carry at least one
 * mechanism or capacitance only.  On success *out owns device memory until
 * cn_model_destroy.  Errors: CN_EINVAL (validation, message in
 * cn_last_error(NULL)), CN_ENOMEM, CN_ECUDA.                               */
cn_status cn_model_create(const cn_morph* morph, const cn_mech_table* mechs, int32_t n_mechs,
                          const cn_options* opt, cn_model** out);

/* NetCon (Table 2): a spike of cell src_gid delivers weight_uS to EXPSYN
 * instance target_syn (index into the EXPSYN table) delay_ms later, rounded
 * to whole steps half away from zero.  The minimum delay over all NetCons
 * sets the spike-exchange interval (Section 2) and must be >= 1 step.
 * Allowed only before the first cn_run (CN_ESTATE after).                  */
cn_status cn_add_netcon(cn_model* m, int32_t src_gid, int32_t target_syn, double weight_uS,
                        double delay_ms);
/* Batch form of cn_add_netcon; NetCon indices follow call order.          */
cn_status cn_add_netcons(cn_model* m, int64_t n, const int32_t* src_gid, const int32_t* target_syn,
                         const double* weight_uS, const double* delay_ms);

/* External events (a kick, Poisson background): event e adds weight_uS[e] to
 * EXPSYN target_syn[e] at step round(t_ms[e]/dt).  Events due at the same
 * step are applied in input order, before NetCon events of that step.
 * Before the first cn_run only (CN_ESTATE after).                          */
cn_status cn_add_events(cn_model* m, int64_t n, const int32_t* target_syn, const double* t_ms,
                        const double* weight_uS);

/* Current clamp: +amp_nA into node (global) while del <= (k+1/2) dt < del+dur.
 * Before the first cn_run only.                                            */
cn_status cn_add_stim(cn_model* m, int32_t node, double del_ms, double dur_ms, double amp_nA);

/* Half gap junctions (gap-junction coupling under the fixed step, Section
 * 3.5; voltages exchanged every time step, Section 5; here they stay on the
 * device): entry i injects g_uS[i] (v(peer[i]) - v(node[i])) nA into
 * node[i], with node[i]'s own voltage implicit and the peer's voltage of
 * the start of the step (voltages are exchanged every step).  A symmetric
 * junction is two entries.  node and peer are global node indices (host
 * arrays, copied).  With any gap junction the exchange interval becomes one
 * step.  Call before the first cn_run.  Errors: CN_EINVAL (range, g < 0),
 * CN_ESTATE.                                                              */
cn_status cn_add_gaps(cn_model* m, int64_t n, const int32_t* node, const int32_t* peer, const double* g_uS);

/* Record the voltage of a node (global index) at every step; *rec_id is the
 * handle for cn_get_trace.  Before the first cn_run only.                  */
cn_status cn_record(cn_model* m, int32_t node, int32_t* rec_id);

/* Advance to step round(tstop_ms/dt) (continuing from the current step).
 * Launches are queued on the model's stream; errors detected on the device
 * (buffer overflow, bounded-wait timeout) are returned by the next call that
 * synchronizes (cn_sync, cn_get_*).  CN_EINVAL if tstop is behind the
 * current time.                                                            */
cn_status cn_run(cn_model* m, double tstop_ms);

/* Wait for queued work and report device-side errors.                      */
cn_status cn_sync(cn_model* m);

/* Current step index k (v holds v_k).                                      */
int64_t cn_current_step(const cn_model* m);

/* Spike raster (Section 3.1: spikes are the simulation's output), sorted by
 * (step, gid).  A spike (gid, k) means the threshold node of cell gid crossed
 * its threshold upward between steps k-1 and k.  Two-call form: with gid or
 * step NULL only *n is set; otherwise at most cap entries are written and *n
 * is the total count (CN_ERANGE if cap < total).                          */
cn_status cn_get_spikes(cn_model* m, int32_t* gid, int64_t* step, size_t cap, size_t* n);

/* Voltage trace of a recorded node: v at steps 0..current (n = current+1).
 * Two-call form as cn_get_spikes.                                          */
cn_status cn_get_trace(cn_model* m, int32_t rec_id, double* out, size_t cap, size_t* n);

/* Every recorded trace at once, step-major: out[k * n_rec + rec_id] for
 * k = 0..step (one contiguous copy; cn_get_trace reads one probe).
 * Two-call: out NULL -> *n = (step + 1) * n_rec.  Errors: CN_ERANGE.     */
cn_status cn_get_traces(cn_model* m, double* out, size_t cap, size_t* n);

/* Node voltages v_k of every node, in global input order (cap >= n_nodes). */
cn_status cn_get_v(cn_model* m, double* out, size_t cap);

/* State column col of mechanism type (HH: 0 m, 1 h, 2 n; EXPSYN: 0 g; channel
 * types: their gates in parameter order; CAHVA: 2 = cai), per instance in
 * table order (cap >= instance count).                                     */
cn_status cn_get_state(cn_model* m, int32_t type, int32_t col, double* out, size_t cap);

/* Number of compartment updates performed so far (sum of cell sizes x steps). */
int64_t cn_updates(const cn_model* m);

/* Diagnostics of the last cn_run: kernel launches issued.                  */
int64_t cn_launch_count(const cn_model* m);

/* Return to step 0: v = v_init, gates at steady state, synaptic g = 0,
 * external-event cursors rewound, spike raster and traces cleared.
 * Parameters set with cn_set_cell_param are kept.                          */
cn_status cn_reset(cn_model* m);

/* Checkpoint / restart of the network (Section 3.4).  A checkpoint holds,
 * in the model's input order (so it restores under any mapping), the state
 * at the current step: every node voltage, every gating state and synaptic
 * conductance, [Ca]i, the threshold flags, and, in place of the undelivered
 * NetCon events, the spike history of the intervals that can still deliver
 * (each delivery is re-derived from its source spike, as the paper collapses
 * pending messages back into the firing event).
 * cn_checkpoint_save: the step must be an interval boundary (a multiple of
 * the minimum NetCon delay).  Two-call: with buf NULL, *n = bytes needed;
 * otherwise writes *n bytes to the HOST buffer buf (cap >= *n).  Errors:
 * CN_ESTATE (not at a boundary), CN_ERANGE (cap too small).
 * cn_checkpoint_load: restores into a model built from the same morphology,
 * mechanism placement and NetCons (checked by a fingerprint; parameters,
 * stimuli and external events may differ), before or after its first run.
 * The model continues from the checkpoint step with its OWN external events
 * and stimuli at and after that step, so a restored network can be driven
 * by new inputs.  Its raster reports spikes after the checkpoint step only;
 * recorded traces start at that step.  Errors: CN_EINVAL (not a checkpoint,
 * another network).                                                        */
cn_status cn_checkpoint_save(cn_model* m, void* buf, size_t cap, size_t* n);
cn_status cn_checkpoint_load(cn_model* m, const void* buf, size_t n);

/* Per-cell maximal conductances (the adjoint's parameters): */
typedef enum {
  CN_PARAM_GNABAR = 0,  /* gnabar of every HH instance of the cell (S/cm2) */
  CN_PARAM_GKBAR = 1,   /* gkbar of every HH instance of the cell (S/cm2)  */
  CN_PARAM_GPAS = 2     /* g of every pas instance of the cell (S/cm2)     */
} cn_cell_param;

/* Set / read one per-cell parameter, values[n_cells] in gid order.  A set
 * takes effect from the next step.                                        */
cn_status cn_set_cell_param(cn_model* m, int32_t param, const double* values);
cn_status cn_get_cell_param(cn_model* m, int32_t param, double* values);

/* Prepare the discrete adjoint of the FP64 run (an extension: the paper has
 * no adjoint): from step 0, cn_run
 * stores the state (v, HH gates, synaptic g) every checkpoint_steps steps.
 * Needs FP64, no NetCons, no external events, at most one HH instance per
 * cell.  Errors: CN_ESTATE, CN_EINVAL.                                     */
cn_status cn_enable_adjoint(cn_model* m, int32_t checkpoint_steps);

/* Gradient of a loss J(traces) with respect to the per-cell parameters
 * above, by the discrete adjoint of the run from step 0 to the current step
 * K: dJ_dtrace is [n_rec][K+1] (host, the derivative of J with respect to
 * every recorded voltage); grad is [3][n_cells] (host; CN_PARAM order).  The
 * reverse pass walks the checkpoint segments backwards, recomputing each
 * segment's trajectory with the forward kernel, and solves the transposed
 * tree system of every step (Hines with the couplings swapped) plus the HH
 * gate sensitivities.  The model's state is left at step K.               */
cn_status cn_run_adjoint(cn_model* m, const double* dJ_dtrace, double* grad);

/* Kernel timing (diagnostics): while enabled, cn_run brackets every
 * interval-kernel and spike-pull launch with CUDA events on the model's
 * stream.  cn_profile_read synchronizes, returns the summed device time (ms)
 * and launch counts since the last read, and clears them.                 */
cn_status cn_profile(cn_model* m, int32_t enable);
cn_status cn_profile_read(cn_model* m, double* interval_ms, int64_t* interval_launches, double* pull_ms,
                          int64_t* pull_launches);

/* Batched tree solve (Section 2: Gaussian elimination in Hines order, as in
 * the per-step matrix resolution).  All arrays are DEVICE pointers of the
 * current device; trees are concatenated: tree t owns rows
 * [offset[t], offset[t+1]) with cell-local parent (parent[first] = -1,
 * 0 <= parent[i] < i - first otherwise).  Row i has diagonal d[i] and
 * coupling b[i] to its parent p; row p has coupling a[i] to i.  Writes the
 * solution to x (which may not alias the inputs); inputs are not modified.
 * offset must satisfy offset[0] = 0, offset[n_trees] = n_nodes and
 * offset[t] <= offset[t+1]; this is checked on the device before any tree is
 * touched, and a violation solves nothing.  Allocates n_nodes doubles of
 * scratch (stream-ordered) per call and synchronizes the stream before
 * returning.  Errors: CN_EINVAL (bad sizes, NULL pointers, bad offsets, or a
 * bad parent index, detected on the device; such a tree is left unsolved),
 * CN_ERANGE (a zero pivot), CN_ENOMEM, CN_ECUDA.                           */
cn_status cn_solve_trees(int32_t n_trees, int64_t n_nodes, const int32_t* offset, const int32_t* parent,
                         const double* a, const double* b, const double* d, const double* rhs, double* x,
                         void* stream);

/* cn_solve_trees without any device allocation.  The paper has no
 * counterpart: this exists for callers that cannot allocate device memory
 * when they solve -- for example because another allocator already reserved
 * the whole GPU, or because an allocation would stall a latency-critical
 * loop.  Same arguments, layout and results as cn_solve_trees, but the
 * working diagonal lives in a fixed array built into the library: at most
 * 1,048,576 rows (n_nodes) per call (CN_ERANGE above that); every GPU that
 * loads the library holds that 8 MiB array until the process exits.  The
 * first call on a device looks up the array's device address (once per
 * device), so make that first call before any stream capture.  That address
 * belongs to the device's primary context: after cudaDeviceReset() of the
 * device it is stale, so do not call this entry point again in a process
 * that reset the device after its first call.  Each call clears its status
 * word first, so an error in one call does not leak into the next.  All calls on
 * a device share the one array: calls whose execution overlaps on the GPU
 * (other streams, other host threads) race and must be serialized by the
 * caller.  Synchronizes the stream before returning; allocates nothing.    */
cn_status cn_solve_trees_noalloc(int32_t n_trees, int64_t n_nodes, const int32_t* offset, const int32_t* parent,
                                 const double* a, const double* b, const double* d, const double* rhs, double* x,
                                 void* stream);

/* Diagnostics: the FP64 rate this GPU attains (TFLOP/s, 2 flops per fused
 * multiply-add) on a stream of independent fused multiply-adds, four warps
 * per SM sub-partition, timed with CUDA events on the model's stream (a
 * scratch buffer comes from the model's allocator).  The interval kernel's
 * FP64 roofline is quoted against it and against the nominal rate.
 * Errors: CN_EINVAL, CN_ENOMEM, CN_ECUDA.                                 */
cn_status cn_fp64_peak(cn_model* m, double* tflops);

/* The reciprocal the engine's solve takes of every pivot (diagnostics):
 * out[i] = 1/d[i] for n DEVICE values d[i] in [2^-1021, 2^1021] (a pivot of
 * the row-scaled cable matrix is >= 1), computed as the interval kernel does
 * -- a float seed refined by Newton-Raphson steps (Markstein's division
 * method) -- instead of an IEEE division; within 1 ulp of the correctly
 * rounded 1/d.  Synchronizes the stream.  Errors: CN_EINVAL, CN_ECUDA.     */
cn_status cn_pivot_reciprocal(int64_t n, const double* d, double* out, void* stream);

/* Error text of the last failed call on m (or of the last failed
 * cn_model_create when m is NULL).  Valid until the next call on m.        */
const char* cn_last_error(const cn_model* m);

/* Release every device buffer of m (through the model's allocator).        */
void cn_model_destroy(cn_model* m);

#ifdef __cplusplus
}
#endif

#endif /* CN_H_ */
