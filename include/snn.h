/*
 * snn.h -- C ABI of the GB300-native on-device network construction and spike
 * delivery library (libsnn.so).
 *
 * The library follows the problem statement of "Scalable Construction of Spiking
 * Neural Networks using up to thousands of GPUs" (arXiv 2512.09502):
 *   - create neuron populations (Results, introduction of the phases: "neuron and
 *     device creation");
 *   - connect them with probabilistic rules (Methods, "Creation of the remote
 *     connection structures for point-to-point MPI communication": Connect /
 *     RemoteConnect(sigma, s, tau, t, p, C, D, alpha));
 *   - calibrate = network construction + "simulation preparation" (Methods,
 *     "Simulation phases and optimization");
 *   - simulate (state propagation), read spikes.
 * The paper's MPI ranks become logical ranks inside one GPU: neurons are distributed
 * round-robin over n_ranks partitions, each rank stores the connections of its
 * targets with image neurons for remote sources, and spikes are routed through the
 * paper's point-to-point (R/L, S, T/P) or collective (H, I, G/Q) maps held in device
 * memory.
 *
 * Conventions for every call:
 *   - returns SNN_OK (0) or a negative SNN_E* status; no exception crosses the ABI;
 *     snn_last_error() gives a message for the last failing call on a context;
 *   - pointers named host_* are host memory owned by the caller; the library copies
 *     into / out of them and synchronises its stream before returning;
 *   - all device memory is owned by the library and comes from the snn_allocator
 *     given at snn_create (or cudaMallocAsync / cudaFreeAsync when it is NULL);
 *   - all device work is issued on the stream given at snn_create;
 *   - global neuron ids (gids) are 0-based in creation order; rank-local indices
 *     appear only in snn_get_connections / snn_get_row / snn_get_maps.
 */
#ifndef SNN_H
#define SNN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes -------------------------------------------------------- */
#define SNN_OK 0
#define SNN_EINVAL (-1)    /* invalid argument or unsupported combination        */
#define SNN_ENOMEM (-2)    /* the allocator returned NULL                        */
#define SNN_ECUDA (-3)     /* a CUDA runtime call or kernel failed               */
#define SNN_ETIMEOUT (-4)  /* a bounded device-side wait gave up                 */
#define SNN_ESTATE (-5)    /* call not valid in the current phase                */
#define SNN_EOVERFLOW (-6) /* a caller buffer or the spike log was too small     */

/* ---- enums --------------------------------------------------------------- */
#define SNN_RULE_FIXED_INDEGREE 0     /* param = K: K sources per target            */
#define SNN_RULE_FIXED_TOTAL 1        /* param = N: N (source, target) draws        */
#define SNN_RULE_PAIRWISE_BERNOULLI 2 /* param = p: each pair kept with prob. p    */
/* param = p: each pair kept with probability p, drawn as geometric gaps between kept
   sources (one draw per kept pair instead of one test per pair; p >= ~5e-6) */
#define SNN_RULE_PAIRWISE_BERNOULLI_GEOMETRIC 3
/* Rules that use every source: one-to-one (target i from source i; needs n_src == n_tgt;
   counter i) and all-to-all (every pair once; counter i_t n_src + i_s).  param is
   ignored.  The threshold xi does not apply to them: they use every source of the
   call, so no flagging decision is taken (Methods, "Remote connections"). */
#define SNN_RULE_ONE_TO_ONE 4
#define SNN_RULE_ALL_TO_ALL 5

#define SNN_W_CONST 0        /* weight = mean                                          */
#define SNN_W_NORMAL_SIGN 1  /* normal(mean, sd), clamped at 0 to keep mean's sign    */
#define SNN_D_CONST 0        /* delay = mean ms, rounded to steps, >= 1 step          */
#define SNN_D_NORMAL_MIN 1   /* normal(mean, sd) ms clipped below at lo, quantised    */

#define SNN_WEIGHT_F32 0   /* stored weights: fp32                                    */
#define SNN_WEIGHT_BF16 1  /* bf16 (round to nearest even of the fp32 draw)           */
#define SNN_WEIGHT_F16 2   /* fp16 of w / scale, scale = power of two per source row  */

#define SNN_EXCHANGE_P2P 0        /* route spikes through T/P packets and L maps  */
#define SNN_EXCHANGE_COLLECTIVE 1 /* route through Q positions and I arrays       */

/* map selectors for snn_get_maps (paper notation) */
#define SNN_MAP_R 0  /* R_{tau,sigma}: remote source local index, ascending (on tau) */
#define SNN_MAP_L 1  /* L_{tau,sigma}: image local index, aligned with R (on tau)    */
#define SNN_MAP_S 2  /* S_{tau,sigma}: source sequence built on sigma (== R)         */
#define SNN_MAP_T 3  /* T_{sigma,s} for every s of sigma, concatenated (CSR values) */
#define SNN_MAP_P 4  /* P_{sigma,s} aligned with T                                   */
#define SNN_MAP_TP_PTR 5 /* CSR offsets of T/P over s = 0..M_sigma (M_sigma+1)       */
#define SNN_MAP_H 6  /* H_{0,sigma}: sorted sources of sigma with a remote image     */
#define SNN_MAP_I 7  /* I_{0,sigma,tau}: image of H[j] in tau or -1                  */
#define SNN_MAP_Q 8  /* Q_{sigma,s} (group 0 only): position of s in H, CSR values   */
#define SNN_MAP_GQ_PTR 9 /* CSR offsets of G/Q over s = 0..M_sigma                   */

/* ---- structs ------------------------------------------------------------- */
typedef struct snn_ctx snn_ctx;

typedef struct snn_allocator {
  /* Return device memory of at least `bytes` bytes usable on `stream`, or NULL.  The
     pointer must be 16-byte aligned (kernels use 16-byte vector accesses); a
     misaligned pointer is released again and the call that asked fails with ENOMEM. */
  void* (*alloc)(void* user, size_t bytes, void* stream);
  /* Release memory obtained from alloc. */
  void (*free)(void* user, void* ptr, size_t bytes, void* stream);
  void* user;
} snn_allocator;

typedef struct snn_config {
  double dt_ms;                /* simulation resolution h in ms (> 0)                 */
  uint32_t n_ranks;            /* logical ranks (>= 1), neurons round-robin            */
  int32_t weight_format;       /* SNN_WEIGHT_*                                         */
  int32_t exchange;            /* SNN_EXCHANGE_* (used when n_ranks > 1)               */
  int32_t use_graph;           /* capture the simulation step as a CUDA graph          */
  uint64_t spike_log_capacity; /* spikes kept for snn_get_spikes; 0 = no recording    */
  int32_t radix_bits;          /* widest sort digit: 8, 9 or 10 (8-bit digits widened
                                  as the key needs); 0 = 10                             */
  int32_t device;              /* CUDA device ordinal                                  */
  int32_t profile_kernels;     /* time every update / deliver launch with CUDA events
                                  (no graph then); results in snn_stats_t.  1: on the
                                  schedule the steps run (one rank: the neuron work and
                                  the delivery of a step overlap on two streams, each
                                  timed on its own stream); 2: the sequential update ->
                                  deliver chain, also on one rank                      */
  int32_t sort_items;          /* records per thread of a sort tile: 8, 12, 16; 0 = tuned */
  int32_t deliver_ctas_per_sm; /* delivery grid = SMs x this (1..32); 0 = tuned          */
  /* Dry run (Results, "Collective communication": each process builds its regular share
     of a larger network in the absence of the rest, to estimate memory and construction
     time): with dry_run = 1 and n_ranks > 1, snn_calibrate builds only the connections,
     image rows and R/L maps of rank dry_run_rank, as if n_ranks ranks existed.  Fixed
     in-degree, one-to-one and all-to-all rules only (EINVAL otherwise); no source-side
     maps and no simulation state:
     snn_simulate, snn_get_spikes and snn_get_state return ESTATE, snn_get_connections /
     snn_get_row / snn_get_maps (R, L) answer for that rank only.  0 = off. */
  int32_t dry_run;
  uint32_t dry_run_rank;
  /* All-sources images (Methods, "Remote connections", threshold xi): a projection whose
     expected connections per source -- K n_target / n_source (fixed in-degree),
     N / n_source (fixed total), p n_target (pairwise Bernoulli) -- reach xi gives every
     one of its sources an image on every rank holding one of its targets, used or not;
     its synapses are then not regenerated for the source-side maps.  Images without
     connections have empty rows.  xi <= 0 (the default) flags used sources only; the
     paper uses xi = 1.  The connections themselves do not depend on xi. */
  double xi;
  int32_t deliver_mode;        /* long rows: 0 = chunks staged in shared memory by bulk
                                  asynchronous copies while earlier chunks are delivered
                                  (when the layout arrays are 16-byte aligned); 1 = each
                                  thread loads its events directly                      */
} snn_config;

/* iaf_psc_exp parameters; potentials in mV relative to E_L = 0, C_m in pF, times in
 * ms, currents in pA.  V0 = V_init_lo, or uniform in [lo, hi) from the VINIT stream
 * when V_init_hi > V_init_lo. */
typedef struct snn_iaf_psc_exp_params {
  double tau_m, C_m, tau_syn_ex, tau_syn_in, V_th, V_reset, t_ref, I_e;
  double V_init_lo, V_init_hi;
  uint64_t v_init_seed;
} snn_iaf_psc_exp_params;

typedef struct snn_rule {
  int32_t kind;  /* SNN_RULE_* */
  double param;  /* K, N or p */
} snn_rule;

typedef struct snn_dist {
  int32_t kind;  /* SNN_W_* for weights, SNN_D_* for delays */
  double mean, sd, lo;
} snn_dist;

typedef struct snn_stats_t {
  uint64_t n_neurons, n_synapses, n_images, n_blocks, n_projections;
  uint64_t n_spikes, n_events, steps_done;   /* since calibrate                 */
  uint64_t device_bytes, peak_device_bytes;  /* through the allocator            */
  uint64_t spike_log_overflow;               /* spikes dropped by a full log    */
  double t_generate_ms, t_sort_ms, t_finalize_ms, t_maps_ms, t_calibrate_ms;
  double t_simulate_ms;
  uint32_t sort_passes, radix_bits, key_bits, ring_slots;
  uint32_t gen_kernel_launches, sort_kernel_launches;
  uint64_t kernel_launches;                  /* library kernels launched so far   */
  uint64_t h2d_bytes, d2h_bytes;             /* host<->device bytes copied so far */
  /* per-kernel CUDA-event times (sort passes always; update / deliver only with
     profile_kernels) and their launch counts */
  double t_sort_pass_ms, t_update_ms, t_deliver_ms;
  uint64_t update_launches, deliver_launches;
} snn_stats_t;

/* ---- lifecycle -----------------------------------------------------------
 * snn_create: new context on config->device; `alloc` may be NULL (cudaMallocAsync);
 * `cuda_stream` is a cudaStream_t (NULL = legacy default stream).  EINVAL on a bad
 * config.  The context owns every device buffer; snn_destroy frees them. */
int snn_create(const snn_config* config, const snn_allocator* alloc, void* cuda_stream,
               snn_ctx** out);
void snn_destroy(snn_ctx* ctx);
const char* snn_last_error(snn_ctx* ctx);

/* ---- construction (before snn_calibrate; ESTATE afterwards) -------------- */

/* Neuron creation ("neuron and device creation" phase): appends n neurons; writes
 * the first new gid to *first_gid. */
int snn_create_population(snn_ctx* ctx, uint32_t n, const snn_iaf_psc_exp_params* params,
                          uint32_t* first_gid);

/* Connect: sources [src_first, src_first + n_src) onto targets [tgt_first,
 * tgt_first + n_tgt) (global ids) with `rule`, weights from `weight` (pA), delays from
 * `delay` (ms).  Multapses and autapses are allowed (fixed in-degree / fixed total),
 * as in the paper's balanced network.  Draws come from Philox-4x32-10 keyed by
 * `seed` and counted per projection, so the network does not depend on n_ranks
 * (the paper's aligned RNG_{sigma,tau} streams, Methods "Point-to-point MPI
 * communication").  Writes the projection id (call order) to *proj_id.  The build is
 * deferred to snn_calibrate so that every projection and rank is built in one batch. */
int snn_connect(snn_ctx* ctx, uint32_t src_first, uint32_t n_src, uint32_t tgt_first,
                uint32_t n_tgt, const snn_rule* rule, const snn_dist* weight,
                const snn_dist* delay, uint64_t seed, uint32_t* proj_id);

/* RemoteConnect(sigma, s, tau, t, p, C, D, alpha) on contiguous rank-local index
 * ranges: sources s_first..s_first+n_s-1 of rank sigma onto targets
 * t_first..t_first+n_t-1 of rank tau (round-robin partition, so the gids are
 * s * n_ranks + sigma: a strided projection of the same generator).  Port p must be
 * 0; alpha is -1 (point-to-point) or 0 (the all-ranks group) -- the maps of both
 * exchange schemes are always built.  EINVAL for ranks or ranges out of bounds. */
int snn_remote_connect(snn_ctx* ctx, uint32_t sigma, uint32_t s_first, uint32_t n_s,
                       uint32_t tau, uint32_t t_first, uint32_t n_t, uint32_t port,
                       const snn_rule* rule, const snn_dist* weight, const snn_dist* delay,
                       int32_t group, uint64_t seed, uint32_t* proj_id);

/* Independent Poisson drive of rate_hz for gids [first, first + n): each input spike
 * adds weight_pA to the synaptic current of the sign's receptor. */
int snn_set_poisson_drive(snn_ctx* ctx, uint32_t first, uint32_t n, double rate_hz,
                          double weight_pA, uint64_t seed);

/* Network construction and simulation preparation on the GPU: connection
 * generation, source/delay sort, per-rank CSR, image neurons and every map, neuron
 * state and propagators (FP64 on the host, stored FP32).  ETIMEOUT if a bounded
 * device wait gave up, ENOMEM / ECUDA as usual.  Call once. */
int snn_calibrate(snn_ctx* ctx);

/* ---- simulation ---------------------------------------------------------- */

/* Advance `steps` steps of dt (state propagation): neuron update, spike routing
 * through the maps, ring-buffer delivery.  Returns after the work is queued and the
 * stream synchronised. */
int snn_simulate(snn_ctx* ctx, uint32_t steps);

/* Copy recorded spikes (step, gid), sorted by (step, gid), into host arrays of
 * capacity `cap`; *n_out = number recorded.  EOVERFLOW if cap is too small (the
 * first cap spikes are written). */
int snn_get_spikes(snn_ctx* ctx, uint32_t* host_step, uint32_t* host_gid, uint64_t cap,
                   uint64_t* n_out);

/* Copy V (mV), I_ex, I_in (pA) of gids [first, first + n) into host arrays (any may be
 * NULL).  When every population has tau_syn_ex == tau_syn_in the two receptors share
 * one ring buffer and one current: I_ex then holds the total synaptic current and I_in
 * is 0 (the membrane dynamics are identical). */
int snn_get_state(snn_ctx* ctx, uint32_t first, uint32_t n, float* host_V, float* host_Iex,
                  float* host_Iin);

/* ---- inspection (parity tests) ------------------------------------------ */

/* Rank `rank`'s connections: row_ptr over its M_rank local rows then its image rows
 * (n_rows + 1 entries, relative to the rank's first synapse), targets as rank-local
 * indices, weights as fp32 (decoded from the stored format), delays in steps.  Any
 * output may be NULL to query sizes only (*n_rows, *n_syn).  EOVERFLOW when a
 * capacity is too small. */
int snn_get_connections(snn_ctx* ctx, uint32_t rank, uint64_t* host_row_ptr,
                        uint64_t row_cap, uint32_t* host_tgt, float* host_w,
                        uint8_t* host_d, uint64_t syn_cap, uint64_t* n_rows,
                        uint64_t* n_syn);

/* One row of rank `rank` (sampled parity at full size). */
int snn_get_row(snn_ctx* ctx, uint32_t rank, uint64_t row, uint32_t* host_tgt, float* host_w,
                uint8_t* host_d, uint64_t cap, uint64_t* n_out);

/* One map (SNN_MAP_*) as int64 values; tau / sigma as in the paper's notation
 * (tau = rank holding the map for R/L/I, sigma = source rank; T/P/H/Q/ptr use
 * sigma only). */
int snn_get_maps(snn_ctx* ctx, uint32_t tau, uint32_t sigma, int32_t which, int64_t* host_buf,
                 uint64_t cap, uint64_t* n_out);

/* Integer CDF table of a projection's quantised-normal delay (thresholds, s_min). */
int snn_get_delay_table(snn_ctx* ctx, uint32_t proj_id, uint32_t* host_thr, uint64_t cap,
                        uint64_t* n_out, uint32_t* s_min);

int snn_stats(snn_ctx* ctx, snn_stats_t* out);

/* Failure-detection self-test: runs the sort's bounded look-back wait against a
 * predecessor status that is never published.  The wait gives up after its spin bound
 * (a fraction of a second) and the call returns SNN_ETIMEOUT; SNN_OK would mean the
 * bound did not trigger, SNN_ECUDA a CUDA failure.  Allocates 4 KB of device memory. */
int snn_selftest_bounded_wait(void* cuda_stream);

/* Ceiling probe of the delivery (a measurement of the GPU, no step of the method).  The
 * delivery of a step adds each event's weight into the target's circular buffer, in the
 * slot d steps after the current one (App. F, the delivery figure's panel c): ring word
 * (n + d) mod D.  Its cost is set by these scattered reductions.  The probe
 * issues `reps` launches of n_events reductions each, at the addresses the delivery uses,
 * and adds zeros, so the ring keeps its values and a later snn_simulate is unaffected.
 *   mode 0: the targets, weights and delays of n_events consecutive synapses of the
 *           layout, streamed exactly as the direct delivery streams a row (weights
 *           multiplied by zero): the delivery without its spike list and rows;
 *   mode 1: the delay of the first synapse of every run of 256 and a target drawn
 *           uniformly from the synapse index by Philox-4x32-10: the reductions alone.
 * Launch r starts at synapse (r * n_events) mod (E - n_events + 1) and uses ring slot
 * offset r mod D; the grid is the delivery's.  *ms_per_launch (host) receives the mean
 * CUDA-event time of one launch on the context's stream (launch gaps included).  One
 * logical rank, after snn_calibrate (ESTATE before it or in a dry run); EINVAL for another
 * mode, n_events of 0 or above the synapse count, or reps of 0. */
int snn_ring_reduction_probe(snn_ctx* ctx, int32_t mode, uint64_t n_events, uint32_t reps,
                             double* ms_per_launch);

/* ---- allocation-free construction ----------------------------------------
 * The paper has no counterpart to this entry point; it serves callers that cannot
 * call cudaMalloc (a host application that owns all device memory under a fixed
 * budget, e.g. a simulator embedding this library as a plugin, or a loop that must
 * never reach the allocator).
 *
 * Builds the source-sorted connections of ONE projection between neurons
 * [0, n_neurons) on one logical rank -- exactly what snn_calibrate builds for a
 * context with n_ranks = 1, one population of n_neurons and this single projection
 * (projection id 0), with fp32 weights -- into caller-owned DEVICE buffers:
 *   dev_row_ptr  uint64[n_neurons + 1]  row starts (row = source gid)
 *   dev_tgt      uint32[syn_cap]        target gid
 *   dev_w        float[syn_cap]         weight (pA)
 *   dev_d        uint8[syn_cap]         delay (steps)
 * *n_syn (host) receives the synapse count.  Rules: fixed in-degree or fixed total.
 * Work is issued on `cuda_stream` (a cudaStream_t) and synchronised before return.
 *
 * Nothing is allocated: no cudaMalloc, cudaFree or allocating library routine.
 * Intermediate data live in a file-scope __device__ scratch array of fixed size,
 * held by every GPU that loads the library until the process exits (about 16.5 MB).
 * The limit: at most SNN_NOALLOC_MAX_SYNAPSES synapses per call; larger requests
 * return SNN_EINVAL.  The first call on a device looks up the scratch array's device
 * address (cudaGetSymbolAddress); make that first call before any stream capture.
 * Every call on a device shares the one scratch array, which keeps the previous
 * call's contents (the call clears what must start at zero): calls that overlap on
 * the GPU (concurrent streams or threads on one device) race and must be serialised
 * by the caller.  Errors: EINVAL (bad arguments or over the limit), EOVERFLOW
 * (syn_cap too small, *n_syn set), ETIMEOUT / ECUDA; a message goes to host_errmsg
 * (may be NULL). */
#define SNN_NOALLOC_MAX_SYNAPSES 1048576ull
int snn_connect_sorted_noalloc(uint32_t n_neurons, uint32_t src_first, uint32_t n_src,
                               uint32_t tgt_first, uint32_t n_tgt, const snn_rule* rule,
                               const snn_dist* weight, const snn_dist* delay, uint64_t seed,
                               double dt_ms, uint64_t* dev_row_ptr, uint32_t* dev_tgt,
                               float* dev_w, uint8_t* dev_d, uint64_t syn_cap, uint64_t* n_syn,
                               void* cuda_stream, char* host_errmsg, size_t errmsg_len);

#ifdef __cplusplus
}
#endif
#endif /* SNN_H */
