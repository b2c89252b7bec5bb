/*
 * abc_gb300.h -- C ABI of the GB300 (sm_103a) library for ABC rejection
 * sampling of the six-compartment stochastic COVID-19 model of
 * Kulkarni, Krell, Nabarro, Moritz, "Hardware-accelerated Simulation-based
 * Inference of Stochastic Epidemiology Models for COVID-19" (2020).
 *
 * The method (paper Sec. 2.1, 2.2, 3.1): draw theta from a uniform prior box
 * (Eq. 1, Eq. 2), simulate the compartments X = [S, I, A, R, D, Ru] (Eq. 3) day
 * by day with the infection rate g (Eq. 4), the hazards h (Eq. 5) and floored
 * Gaussian transition counts, compare the simulated (A, R, D) series with the
 * observed one by Euclidean distance and accept theta when the distance is at
 * most eps (Eq. 7); all samples are independent (Sec. 3.1).
 *
 * Conventions shared by every entry point
 *  - theta layout: [alpha0, alpha, n, beta, gamma, delta, eta, kappa] (Eq. 1).
 *  - observed: HOST int32 array [3][T+1], row-major, rows A, R, D. Column 0 is the
 *    initial condition (A0, R0, D0); columns 1..T are compared with days 1..T.
 *    Entries must be >= 0 and A0 + R0 + D0 <= N_pop.
 *  - N_pop: total population P, 1 <= P < 2^31 (compartments are int32).
 *  - T: simulated days, 1 <= T <= ABC_T_MAX.
 *  - Random numbers: Philox4x32-10 keyed by seed; sample index i, day-pair k and
 *    block g form the counter (i_lo, i_hi, k, 4*stream + g); stream < 2^30.
 *    Results therefore depend only on (seed, stream, i), never on the launch
 *    shape, so any split of the index range reproduces the unsplit run.
 *  - mode: ABC_EXACT uses the library's fixed float32 series for log2, exp2,
 *    sin(pi x), cos(pi x) and IEEE-rounded +, -, *, /, sqrt with no FMA
 *    contraction (bit-reproducible); ABC_FAST uses the GPU's approximate
 *    transcendental units and FMA (same random numbers, statistically equivalent).
 *  - Device pointers are CUDA device memory of the current device; they are owned
 *    by the caller. cuda_stream is a cudaStream_t (NULL = legacy default stream).
 *    Every call is stream-ordered on cuda_stream; calls that return host results
 *    (n_accepted, eps) synchronize that stream before returning.
 *  - Scratch that a call allocates stream-ordered comes from a memory pool the
 *    library creates on each device's first use; it keeps up to 1 GiB of freed
 *    scratch mapped for later calls (more is given back at synchronisations).
 *  - Errors: every call returns an abc_status. On error, abc_last_error() gives a
 *    thread-local message. No C++ exception crosses this boundary.
 */
#ifndef ABC_GB300_H
#define ABC_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ABC_T_MAX 4096
#define ABC_STREAM_MAX ((1u << 30) - 1u)

/* Uniform prior box (Sec. 2.1, Eq. 2): theta_j = lo_j + (hi_j - lo_j) u_j.
 * The paper's box is lo = 0, hi = {1, 100, 2, 1, 1, 1, 1, 2}. Bounds must be
 * finite with lo_j <= hi_j. */
typedef struct {
    float lo[8];
    float hi[8];
} abc_prior_box;

/* Arithmetic mode. ABC_EXACT: the library's own fixed FP32 series for log2,
 * exp2, sin and cos, every operation IEEE round-to-nearest and no FMA
 * contraction, so results equal a plain CPU implementation bit for bit.
 * ABC_FAST: the SFU approximations and FMA, judged statistically.
 * ABC_VARIANCE_LITERAL may be OR-ed into either for the model variant that
 * reads the transition variance of Sec. 2.1 literally (standard deviation
 * h^(1/4) instead of sqrt(h)); it is accepted by abc_sample, abc_sample_async,
 * abc_sample_noalloc, abc_distances, abc_simulate, abc_step and abc_project,
 * and rejected (ABC_ERR_INVALID_ARG) by the batched and sequential calls. */
typedef enum { ABC_EXACT = 0, ABC_FAST = 1, ABC_VARIANCE_LITERAL = 4 } abc_mode;

typedef enum {
    ABC_OK = 0,
    ABC_ERR_INVALID_ARG = 1, /* an argument is out of range or a pointer is NULL */
    ABC_ERR_CAPACITY = 2,    /* more accepts than the output capacity */
    ABC_ERR_CUDA = 3,        /* a CUDA runtime call or a kernel launch failed */
    ABC_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up */
    ABC_ERR_NOMEM = 5        /* device memory allocation failed */
} abc_status;

/* ABC rejection over the sample indices [first_index, first_index + n_samples)
 * (Sec. 2.2 and Sec. 3.1): for each i, draw theta_i from the prior, simulate T
 * days, dist_i = sqrt(sum over days 1..T of the squared (A, R, D) differences),
 * accept when dist_i <= eps.
 *
 *  theta_out  DEVICE float  [capacity][8]   accepted theta
 *  dist_out   DEVICE double [capacity]      accepted distances
 *  idx_out    DEVICE uint64 [capacity]      accepted sample indices
 *  n_accepted HOST   uint64                 number of accepted samples
 *
 * The accepted samples are written in an unspecified order (sort by idx_out for
 * a canonical order). If more than `capacity` samples are accepted the call
 * returns ABC_ERR_CAPACITY, *n_accepted holds the true count and the output
 * buffers hold an unspecified subset of `capacity` accepted samples.
 * Samples whose running distance^2 exceeds eps^2 are abandoned early (partial
 * sums only grow); the result is that of simulating all T days of every sample.
 * Uses a small amount of device scratch memory (the observed series and three
 * counters) and pinned host memory to stage it, allocated on the first call of
 * each host thread on each device, grown when a longer series needs more and
 * kept for the life of the thread. The call synchronises cuda_stream before it
 * returns. Requires eps >= 0 (not NaN) and first_index + n_samples < 2^64. */
abc_status abc_sample(const abc_prior_box* prior, const int32_t* observed, int32_t T,
                      int64_t N_pop, double eps, uint64_t n_samples, uint64_t seed,
                      uint32_t stream, abc_mode mode, uint64_t first_index, float* theta_out,
                      double* dist_out, uint64_t* idx_out, uint64_t capacity,
                      uint64_t* n_accepted, void* cuda_stream);

/* A region's observed series, checked and copied to device memory once, for
 * repeated asynchronous sampling (abc_sample_async). observed is HOST int32
 * [3][T+1] as for abc_sample; the handle keeps a device copy and the initial
 * condition (column 0). Create and destroy synchronise the current device; a
 * handle belongs to the device that was current at creation. */
typedef struct abc_observed_s* abc_observed;
abc_status abc_observed_create(const int32_t* observed, int32_t T, int64_t N_pop, abc_observed* out);
abc_status abc_observed_destroy(abc_observed obs);

/* abc_sample without a host round trip (Sec. 2.2 and Sec. 3.1; the same kernel,
 * accept set and outputs), for pipelined chunks of one region: the call zeroes
 * counters_dev (DEVICE uint64 [3]) on cuda_stream, enqueues the kernel and
 * returns without synchronising. When the stream reaches that point,
 * counters_dev[0] holds the number of accepted samples (the true count, which
 * may exceed capacity: then the outputs hold an unspecified subset of
 * `capacity` of them), counters_dev[1] the kernel's claim counter (index
 * chunks are claimed 32 at a time, so it ends at or above n_samples) and
 * counters_dev[2] the number of model days simulated.
 * Outputs and counters must stay untouched until then. Allocates nothing and
 * may be captured in a CUDA graph. Errors reported are argument errors and
 * launch failures; the capacity check is the caller's. */
abc_status abc_sample_async(const abc_prior_box* prior, abc_observed obs, double eps, uint64_t n_samples,
                            uint64_t seed, uint32_t stream, abc_mode mode, uint64_t first_index,
                            float* theta_out, double* dist_out, uint64_t* idx_out, uint64_t capacity,
                            uint64_t* counters_dev, void* cuda_stream);

/* Rejection sampling until a target number of accepts (Sec. 2.2: draws are
 * repeated until the target number of posterior samples is accepted; Sec. 3.1:
 * each iteration is one vectorised batch). Runs batches of `batch` consecutive
 * sample indices from first_index on, one launch of abc_sample's kernel each
 * on the resident observed series, until at least n_target samples are
 * accepted or max_samples indices are used. The accepted set is every sample
 * accepted among [first_index, first_index + *n_used): the batches are whole
 * (only max_samples may cut the last one), so the set depends on the inputs
 * alone, not on timing. Outputs as abc_sample (DEVICE buffers of `capacity`
 * rows, order unspecified); *n_accepted (HOST) may exceed n_target by the last
 * batch's accepts, and falls short of it only when max_samples ran out.
 * Returns ABC_ERR_CAPACITY as soon as the accepts exceed capacity
 * (*n_accepted, *n_used: the true counts so far; output contents then
 * unspecified). n_target = 0 or max_samples = 0 runs nothing. Synchronises
 * cuda_stream after every batch (one 24-byte read of the counters);
 * abc_last_simulated_days reports the days of all batches. */
abc_status abc_sample_until(const abc_prior_box* prior, abc_observed obs, double eps, uint64_t n_target,
                            uint64_t batch, uint64_t max_samples, uint64_t seed, uint32_t stream, abc_mode mode,
                            uint64_t first_index, float* theta_out, double* dist_out, uint64_t* idx_out,
                            uint64_t capacity, uint64_t* n_accepted, uint64_t* n_used, void* cuda_stream);

/* The distance of every sample in [first_index, first_index + n_samples)
 * (Sec. 2.2): dist_out DEVICE double [n_samples], dist_out[j] the distance of
 * sample first_index + j. theta_out, when not NULL, is DEVICE float
 * [n_samples][8] and receives each sample's prior draw. Asynchronous on
 * cuda_stream. Uses device scratch for the observed series like abc_sample. */
abc_status abc_distances(const abc_prior_box* prior, const int32_t* observed, int32_t T,
                         int64_t N_pop, uint64_t n_samples, uint64_t seed, uint32_t stream,
                         abc_mode mode, uint64_t first_index, double* dist_out,
                         float* theta_out, void* cuda_stream);

/* Trajectories for given parameter vectors (Sec. 2.1): for b < B, simulate
 * theta[b] with the random numbers of sample index sample_index[b] from the
 * initial condition init_ard (HOST int32 [3] = A0, R0, D0) and write
 * traj_out[b][d][c], d = 0..T, c = S, I, A, R, D, Ru.
 *  theta        DEVICE float  [B][8]
 *  sample_index DEVICE uint64 [B]
 *  traj_out     DEVICE int32  [B][T+1][6]
 * A sample accepted by abc_sample, replayed with its (theta, idx), reproduces
 * the trajectory whose distance was reported. Asynchronous on cuda_stream. */
abc_status abc_simulate(const float* theta, const uint64_t* sample_index, uint64_t B,
                        const int32_t* init_ard, int32_t T, int64_t N_pop, uint64_t seed,
                        uint32_t stream, abc_mode mode, int32_t* traj_out, void* cuda_stream);

/* One model day (Sec. 2.1, second to fourth step) applied to B given states:
 * state_in[b] (S, I, A, R, D, Ru) with theta[b], using the five normals of day
 * day[b] (>= 1) of sample sample_index[b]. Writes state_out[b] and the five
 * transition counts counts_out[b] (S->I, I->A, A->R, A->D, I->Ru).
 *  theta DEVICE float [B][8]; state_in, state_out DEVICE int32 [B][6];
 *  sample_index DEVICE uint64 [B]; day DEVICE int32 [B]; counts_out DEVICE
 *  int32 [B][5] or NULL. States must be >= 0 with sum N_pop. Asynchronous. */
abc_status abc_step(const float* theta, const int32_t* state_in, const uint64_t* sample_index,
                    const int32_t* day, uint64_t B, int64_t N_pop, uint64_t seed, uint32_t stream,
                    abc_mode mode, int32_t* state_out, int32_t* counts_out, void* cuda_stream);

/* The k-th smallest (1-based, 1 <= k <= n) of n non-negative distances
 * (DEVICE double [n], e.g. from abc_distances), returned in *eps_out (HOST).
 * Used to set eps to a distance quantile. +infinity is allowed; any NaN,
 * negative value or -0 returns ABC_ERR_INVALID_ARG (their bit patterns do not
 * order like values). Synchronizes cuda_stream. Uses device scratch (a
 * histogram) allocated stream-ordered and freed before returning. */
abc_status abc_kth_smallest(const double* dist, uint64_t n, uint64_t k, double* eps_out,
                            void* cuda_stream);

/* The accept step of ABC rejection (Sec. 2.2: accept when the distance is at
 * most eps) on distances already computed, e.g. by abc_distances over the
 * sample indices [first_index, first_index + n): sample j is accepted iff
 * dist[j] <= eps, and its index first_index + j, its distance and, if theta is
 * not NULL, its theta are written out. With dist and theta from abc_distances
 * the accepted set is exactly that of abc_sample with the same arguments and
 * eps; choosing eps as a distance quantile (abc_kth_smallest) and selecting
 * below it costs no second simulation.
 *
 *  dist       DEVICE double [n]             distances of samples 0..n-1
 *  theta      DEVICE float  [n][8] or NULL  their parameters
 *  theta_out  DEVICE float  [capacity][8]   accepted theta (ignored when theta is NULL)
 *  dist_out   DEVICE double [capacity]      accepted distances
 *  idx_out    DEVICE uint64 [capacity]      accepted sample indices
 *  n_selected HOST   uint64                 number of accepted samples
 *
 * Order of the outputs, capacity overflow (ABC_ERR_CAPACITY with the true
 * count in *n_selected) and eps (>= 0, not NaN) as in abc_sample. A NaN
 * distance is never accepted. Uses one stream-ordered scratch counter and
 * synchronises cuda_stream before it returns. */
abc_status abc_select_below(const double* dist, const float* theta, uint64_t n, double eps, uint64_t first_index,
                            float* theta_out, double* dist_out, uint64_t* idx_out, uint64_t capacity,
                            uint64_t* n_selected, void* cuda_stream);

/* ABC rejection with eps at a distance quantile, in one call (Sec. 2.2: a
 * sample is accepted when its distance is at most eps; here eps is the k-th
 * smallest distance among the n_samples samples [first_index, first_index +
 * n_samples), 1 <= k <= n_samples <= 2^40). Computes every distance, eps, and
 * the samples with distance <= eps (at least k; more where distances tie at
 * eps): the same eps and accepted set as abc_distances, abc_kth_smallest and
 * abc_select_below called in turn with the same arguments, with the three
 * steps back to back on the device, one synchronisation, and no distance
 * copied to the host.
 *
 *  theta_out  DEVICE float  [capacity][8]   accepted theta
 *  dist_out   DEVICE double [capacity]      accepted distances
 *  idx_out    DEVICE uint64 [capacity]      accepted sample indices
 *  eps_out    HOST   double                 the k-th smallest distance
 *  n_accepted HOST   uint64                 number of accepted samples
 *
 * Order of the outputs and capacity overflow (ABC_ERR_CAPACITY with the true
 * count in *n_accepted) as in abc_sample. Device scratch: every distance and
 * prior draw (40 bytes per sample, stream-ordered, freed before returning),
 * and the per-thread cached scratch of abc_sample for the series and counters.
 * Synchronizes cuda_stream. */
abc_status abc_sample_quantile(const abc_prior_box* prior, const int32_t* observed, int32_t T,
                               int64_t N_pop, uint64_t n_samples, uint64_t k, uint64_t seed,
                               uint32_t stream, abc_mode mode, uint64_t first_index,
                               float* theta_out, double* dist_out, uint64_t* idx_out,
                               uint64_t capacity, double* eps_out, uint64_t* n_accepted,
                               void* cuda_stream);

/* Posterior-predictive projection (Sec. 5: accepted samples simulated forward
 * for 120 days, plotted as 5th to 95th percentile bands). For b < B simulate
 * theta[b] (DEVICE float [B][8]) with the random numbers of sample_index[b]
 * (DEVICE uint64 [B]) from init_ard (HOST int32 [3]) for T days, then for every
 * day d = 0..T and observed compartment c = A, R, D (0, 1, 2) write the
 * q-quantiles of the B simulated values: bands_out[k][d][c] (DEVICE float
 * [n_q][T+1][3]) = the floor(q_k (B - 1))-th smallest (order statistic,
 * 0-based). quantiles: HOST double [n_q] in [0, 1]. 1 <= B <= 8192. Uses
 * stream-ordered device scratch for the trajectories. Async on cuda_stream. */
#define ABC_PROJECT_MAX_B 8192
abc_status abc_project(const float* theta, const uint64_t* sample_index, uint64_t B, const int32_t* init_ard,
                       int32_t T, int64_t N_pop, uint64_t seed, uint32_t stream, abc_mode mode,
                       const double* quantiles, int32_t n_q, float* bands_out, void* cuda_stream);

/* ------------------------------------------------------------------------
 * Batched regions (many regions, one persistent launch, CUDA-graph replay)
 * ------------------------------------------------------------------------
 * A plan holds up to ABC_MAX_REGIONS regions, each with its own observed
 * series, population, horizon, eps, random stream, sample range and accepted
 * buffers, and runs ABC rejection (the same method and results as abc_sample,
 * region by region) over all of them in one kernel launch. The plan owns all
 * device memory it needs; abc_plan_run allocates nothing and does not
 * synchronize, so it can be captured in a CUDA graph (abc_plan_run_graph does
 * that). Accepted samples accumulate in the plan's buffers across runs until
 * abc_plan_reset. */
#define ABC_MAX_REGIONS 32

typedef struct {
    const int32_t* observed; /* HOST int32 [3][T+1], rows A, R, D (copied at plan creation) */
    int32_t T;               /* simulated days, 1..ABC_T_MAX */
    int64_t N_pop;           /* population, 1 <= N_pop < 2^31 */
    double eps;              /* tolerance, >= 0 */
    uint64_t n_samples;      /* samples per run */
    uint64_t first_index;    /* sample index of the first run; each run advances it by n_samples */
    uint32_t stream;         /* RNG stream of this region (< 2^30) */
    uint64_t capacity;       /* accepted samples kept by the plan for this region */
    const float* theta_in;   /* DEVICE float [n_samples][8] proposals, or NULL to draw from the prior;
                                a proposal whose first coordinate is NaN is skipped (not simulated) */
} abc_region;

typedef struct abc_plan_s* abc_plan;

typedef struct {
    int32_t block_threads;        /* 128, 256 or 512 */
    int32_t pairs_per_iteration;  /* day pairs per loop iteration: 1 or 2 */
    int32_t blocks_per_sm;        /* resident blocks per SM requested (0 = all that fit) */
    int32_t lean;                 /* 1: the kernel form that reads each region's constants from
                                     shared memory where it uses them (64 registers, four
                                     256-thread blocks per SM; fast mode only) */
    float ms;                     /* measured time of one run with this shape */
} abc_launch_shape;

/* Create a plan for n_regions regions (1..ABC_MAX_REGIONS) sharing the prior
 * box, the seed and the arithmetic mode. Allocates the plan's device memory
 * (region table, observed series, counters, accepted buffers) on the current
 * device and copies the observed series. The launch shape starts at 256
 * threads, one day pair per iteration. */
abc_status abc_plan_create(const abc_prior_box* prior, const abc_region* regions, int32_t n_regions,
                           uint64_t seed, abc_mode mode, abc_plan* plan_out);

/* Zero the accepted and simulated-day counters of every region (async). */
abc_status abc_plan_reset(abc_plan plan, void* cuda_stream);

/* One run: every region's n_samples samples from its current first_index, then
 * each first_index advances by n_samples. Async on cuda_stream; no allocation,
 * no synchronization; capturable in a CUDA graph. */
abc_status abc_plan_run(abc_plan plan, void* cuda_stream);

/* n_runs consecutive runs replayed from a CUDA graph that the plan captures
 * on cuda_stream the first time it is called with this n_runs (cuda_stream
 * must then be a non-default stream). Async. */
abc_status abc_plan_run_graph(abc_plan plan, int32_t n_runs, void* cuda_stream);

/* Autotuner: time one run with every launch shape the library is compiled
 * for, keep the fastest, then restore the plan's sample ranges and counters.
 * Synchronizes cuda_stream. shapes_out (HOST, may be NULL) receives up to
 * max_shapes measured shapes; *best_out (may be NULL) the chosen one. */
abc_status abc_plan_tune(abc_plan plan, void* cuda_stream, abc_launch_shape* shapes_out, int32_t max_shapes,
                         int32_t* n_shapes_out, abc_launch_shape* best_out);

/* Accepted samples of one region (synchronizes cuda_stream). *n_accepted is the
 * count since the last reset (may exceed the capacity; the buffers then hold
 * an unspecified subset of `capacity` of them); *simulated_days the model days
 * simulated. theta_out/dist_out/idx_out receive the plan's DEVICE buffers
 * ([capacity][8] float, [capacity] double, [capacity] uint64), owned by the
 * plan and valid until abc_plan_destroy; any of the four may be NULL. */
abc_status abc_plan_results(abc_plan plan, int32_t region, uint64_t* n_accepted, uint64_t* simulated_days,
                            float** theta_out, double** dist_out, uint64_t** idx_out, void* cuda_stream);

/* Copy min(count, accepted, capacity) accepted samples of one region into
 * caller buffers (device or pinned host: cudaMemcpyDefault), async on
 * cuda_stream. theta_dst [count][8] float, dist_dst [count] double,
 * idx_dst [count] uint64; any may be NULL. *copied (HOST, may be NULL) receives
 * the number copied; the call synchronizes to read the count. */
abc_status abc_plan_copy_results(abc_plan plan, int32_t region, float* theta_dst, double* dist_dst,
                                 uint64_t* idx_dst, uint64_t count, uint64_t* copied, void* cuda_stream);

/* Point a region at a new proposal buffer (DEVICE [n_samples][8]) or NULL for
 * prior draws, and/or set its next first_index. Synchronous (cudaMemcpy of the
 * region table, which is not ordered with the plan's stream): no run of the
 * plan may be in flight, so synchronize its stream first. */
abc_status abc_plan_set_region(abc_plan plan, int32_t region, const float* theta_in, uint64_t first_index);

/* Use one of the compiled launch shapes (as abc_plan_tune reports them; ms is
 * ignored) for the following runs, without tuning. A new plan starts with
 * {256 threads, 2 day pairs, lean} in ABC_FAST and {256, 1, standard} in
 * ABC_EXACT. Returns ABC_ERR_INVALID_ARG
 * for a shape the library is not compiled for, or a lean shape in exact mode.
 * Every shape gives the same accepted samples and day counts. As for
 * abc_plan_set_region, no run of the plan may be in flight. */
abc_status abc_plan_set_shape(abc_plan plan, const abc_launch_shape* shape);

/* Set a region's tolerance for the following runs (eps >= 0, not NaN).
 * Synchronous (cudaMemcpy of the one table field); as for
 * abc_plan_set_region, no run of the plan may be in flight. */
abc_status abc_plan_set_eps(abc_plan plan, int32_t region, double eps);

/* Release the plan's device memory and graph. Leaves abc_last_error() as it was. */
abc_status abc_plan_destroy(abc_plan plan);

/* ------------------------------------------------------------------------
 * Learned proposal for sequential ABC: a masked autoregressive flow (MAF)
 * ------------------------------------------------------------------------
 * The paper's Sec. 2.2 points to sequential Monte Carlo ABC: a decreasing
 * sequence of tolerances, each round built from the previous round's
 * accepted samples. The library's proposal for the next round is a density
 * q(theta) on the prior box, learned from the previous round's accepted,
 * importance-weighted samples:
 *  - y = logit((theta - lo) / (hi - lo)) (support = the box);
 *  - n_blocks MADE blocks (one hidden ReLU layer of `hidden` units; output j
 *    depends on inputs < j), each x -> z = (x - mu(x)) exp(-alpha(x)) with
 *    alpha = 6 tanh(alpha_raw / 6), the order reversed between blocks;
 *  - base: independent standard logistic coordinates,
 *    log p(z) = sum_j (-|z_j| - 2 log(1 + exp(-|z_j|))): the logit of a uniform
 *    variable is standard logistic, so with zero parameters q is exactly the
 *    uniform prior, and flat posterior directions keep the prior's tails;
 *  - log q(theta) = log p(z) - sum alpha - sum_j log((hi_j - lo_j) s_j (1 - s_j)),
 *    s = sigmoid(y).
 * Weights live in FP32 (the master copy trained by Adam) and in masked BF16
 * copies used by tensor-core products (mma.sync m16n8k8 / m16n8k16 BF16 with
 * FP32 accumulation). Activations entering a product are rounded to BF16;
 * everything else is FP32.
 *
 * Parameter order (host float arrays): for each block b = 0..n_blocks-1:
 *   W1 [hidden][8] row-major, b1 [hidden], W2 [16][hidden] row-major
 *   (rows 0..7 mu, 8..15 alpha_raw), b2 [16].
 * Masked entries (W1[l][j] with (l mod 7) + 1 < j + 1, W2[o][l] with
 * (o mod 8) + 1 <= (l mod 7) + 1) are ignored. */
typedef struct abc_maf_s* abc_maf;

/* Create a flow with n_blocks (1..4) blocks of `hidden` units (a multiple of
 * 16, 16..256) on the prior box, parameters zero (q = the uniform prior).
 * Allocates its device memory on the current device. The training kernel
 * stages a CTA's operands in shared memory, n_blocks (100 hidden + 192) +
 * 36864 bytes (published BF16 operands per block, tensor-core operand slots
 * of four warps), and its gradient sums in tensor memory: a shape beyond the
 * device's per-block limit returns ABC_ERR_INVALID_ARG (on GB300, 227 KB:
 * every shape up to 4 blocks of 256 fits). */
abc_status abc_maf_create(int32_t n_blocks, int32_t hidden, const abc_prior_box* box, abc_maf* maf_out);

/* A set of n_flows (1..ABC_MAF_MAX_FLOWS) independent flows of the same shape
 * in one object, one per region of a batched run: their parameters sit one
 * flow after another, abc_maf_train_flows trains all of them in the same
 * launches, and the *_at calls sample or evaluate one of them. An object made
 * by abc_maf_create is a set of one flow; the calls without a flow index act
 * on flow 0, except set/get/init, which cover every flow. */
#define ABC_MAF_MAX_FLOWS 64
abc_status abc_maf_create_multi(int32_t n_flows, int32_t n_blocks, int32_t hidden, const abc_prior_box* box,
                                abc_maf* maf_out);
int32_t abc_maf_flow_count(abc_maf maf);

/* Broadened proposal: sampling and density evaluation (abc_maf_sample*,
 * abc_maf_log_q*) use the base z = tau * (standard logistic), density
 * sum_j (log p(z_j / tau) - log tau), for every flow of the object; training
 * still fits the flow with tau = 1 (maximum likelihood). tau in [0.5, 4],
 * default 1. A proposal fitted by maximum likelihood to its own weighted
 * output tends to miss the target's tails round after round, which leaves the
 * self-normalised estimates of a finite run biased toward the proposal's
 * bulk; a base broader than the fitted one keeps covering them. */
abc_status abc_maf_set_proposal_scale(abc_maf maf, float tau);

/* Testing hook for the gradient kernel's bounded waits. With hold != 0 the
 * thread that issues the kernel's tensor-core products issues none, so the
 * kernel's final wait for them runs out (after 2 s): abc_maf_gradient and the
 * training calls then return ABC_ERR_TIMEOUT and leave the flow's gradient
 * unspecified. hold = 0 (the default) restores normal operation; the CUDA
 * context stays usable throughout. Applies to launches after the call (a
 * captured training step is rebuilt). */
abc_status abc_maf_test_hold_products(abc_maf maf, int32_t hold);

/* Random initial parameters: W1 ~ N(0, scale^2 / 8), W2 ~ N(0, scale^2 / hidden),
 * zero biases (so the ReLU units start active and the flow near the base
 * density), from a host generator seeded with `seed`; resets Adam. */
abc_status abc_maf_init_random(abc_maf maf, uint64_t seed, float scale);

/* Number of parameters (floats) of one flow, in the order above. */
int64_t abc_maf_param_count(abc_maf maf);

/* Copy parameters from / to HOST float arrays [n_flows][param_count]
 * (synchronous). Setting parameters also resets the Adam moments. The random
 * initialisation draws the flows one after another from the one generator. */
abc_status abc_maf_set_params(abc_maf maf, const float* params);
abc_status abc_maf_get_params(abc_maf maf, float* params);

/* Draw n proposals: standard logistic base draws u (DEVICE float [n][8], or
 * NULL to draw them with Philox from (seed, stream, i = first_index + j):
 * coordinate c of sample j takes word c mod 4 of the block with counter
 * (i_lo, i_hi, 0, 4 stream + c / 4), whose uniform (2m + 1) 2^-24 (m its low
 * 23 bits) gives the draw log(u / (1 - u))), the sequential
 * inverse of the flow, theta = lo + (hi - lo) sigmoid(y). theta_out DEVICE
 * float [n][8]; logq_out DEVICE float [n] (log q(theta)) or NULL. Async. */
abc_status abc_maf_sample(abc_maf maf, uint64_t n, const float* base_draws, uint64_t seed, uint32_t stream,
                          uint64_t first_index, float* theta_out, float* logq_out, void* cuda_stream);
abc_status abc_maf_sample_at(abc_maf maf, int32_t flow, uint64_t n, const float* base_draws, uint64_t seed,
                             uint32_t stream, uint64_t first_index, float* theta_out, float* logq_out,
                             void* cuda_stream);

/* log q(theta) for n points (DEVICE float [n][8] inside the box) into logq_out
 * (DEVICE float [n]). Async. */
abc_status abc_maf_log_q(abc_maf maf, uint64_t n, const float* theta, float* logq_out, void* cuda_stream);
abc_status abc_maf_log_q_at(abc_maf maf, int32_t flow, uint64_t n, const float* theta, float* logq_out,
                            void* cuda_stream);

/* Gradient of the weighted mean of -log q_y(y(theta)) over n points (theta
 * DEVICE [n][8], weights DEVICE [n] >= 0 or NULL for all ones) into the flow's
 * gradient buffer; *loss_out (HOST, may be NULL) gets the loss. Synchronizes
 * cuda_stream. grads_out (HOST, may be NULL) receives the gradient in the
 * parameter order. The gradient kernel's waits between its warps and the
 * thread that issues its tensor-core products are bounded (2 s each);
 * ABC_ERR_TIMEOUT reports one that ran out, here and in the training calls. */
abc_status abc_maf_gradient(abc_maf maf, uint64_t n, const float* theta, const float* weights, float* loss_out,
                            float* grads_out, void* cuda_stream);

/* One Adam step (Kingma and Ba) of the master parameters with the flow's
 * current gradient, then refresh the BF16 copies; flows of a set whose
 * current gradient has no points keep their parameters. Async. */
abc_status abc_maf_adam_step(abc_maf maf, float lr, float beta1, float beta2, float eps, void* cuda_stream);

/* Weighted maximum-likelihood training: n_steps Adam steps, each on a batch of
 * `batch` rows drawn with replacement (Philox, seed) from the n points
 * (theta DEVICE [n][8], weights DEVICE [n] or NULL). The steps are captured in
 * a CUDA graph and replayed. *loss_out (HOST, may be NULL) gets the full-data
 * loss after training. Synchronizes cuda_stream (a non-default stream is
 * required for the graph). */
abc_status abc_maf_train(abc_maf maf, uint64_t n, const float* theta, const float* weights, int32_t n_steps,
                         int32_t batch, float lr, uint64_t seed, float* loss_out, void* cuda_stream);

/* abc_maf_train for every flow of a set at once, each on its own data: HOST
 * arrays [n_flows] of DEVICE pointers theta[r] ([n[r]][8]) and weights[r]
 * ([n[r]] or NULL; `weights` itself may be NULL for all ones) and of counts
 * n[r] < 2^32; a flow with n[r] = 0 is left as it is. Each step draws `batch`
 * rows per flow and updates all flows with one gradient launch (one CTA row of
 * the grid per flow) and one Adam launch. With val_fraction in (0, 0.5], the
 * last min(floor(val_fraction n[r]), 8192) points of each flow with
 * n[r] >= 20 are held out: every 25 steps each flow's validation loss is measured, a flow keeps
 * the parameters of its best validation loss and stops training after three
 * checks without improvement (early stopping against overfitting a small
 * round); n_steps is then an upper bound. loss_out HOST float [n_flows] or
 * NULL: the kept validation loss (with validation) or the full-data loss.
 * Synchronizes cuda_stream (non-default). */
abc_status abc_maf_train_flows(abc_maf maf, const float* const* theta, const float* const* weights, const uint64_t* n,
                               int32_t n_steps, int32_t batch, float lr, uint64_t seed, float val_fraction,
                               float* loss_out, void* cuda_stream);

/* Release the flow's device memory and captured training step. Leaves
 * abc_last_error() as it was. */
abc_status abc_maf_destroy(abc_maf maf);

/* Sequential ABC with the learned proposal (the SMC-ABC idea of Sec. 2.2):
 * round r simulates sims_per_round proposals at tolerance
 * eps_r = eps0 * eps_factor^r. Round 0 draws from the prior. After each round
 * the flow is trained (weighted maximum likelihood) on that round's accepted
 * samples with importance weights w = prior(theta) / q(theta) (w = 1 for
 * prior draws), and the next round draws from the flow unless fallback_rule
 * sends it back to the prior (ESS = (sum w)^2 / sum w^2; by default when the
 * flow gave fewer effective samples per simulation than the prior's
 * acceptance rate, measured on the round's defensive draws as
 * n_defensive_accepted / n_defensive). Training holds out val_fraction of the round's
 * accepts and stops early (abc_maf_train_flows). A flow round draws a fraction `defensive` of its
 * proposals from the prior and weights every proposal by the mixture density
 * q_mix = (1 - defensive) q + defensive * prior (defensive importance sampling,
 * Hesterberg 1995), so w = prior / q_mix <= 1 / defensive.
 * Accepted draws keep their weights, so the weighted
 * accepted samples of every round estimate the ABC posterior at its
 * tolerance (Eq. 7). Simulations use (seed, stream 0, index r *
 * sims_per_round + j); flow draws use (seed, stream 1, the same index). */
typedef struct {
    int32_t rounds;           /* >= 1 */
    uint64_t sims_per_round;  /* proposals simulated per round */
    double eps0;              /* tolerance of round 0 */
    double eps_factor;        /* in (0, 1] */
    double ess_min;           /* fraction, e.g. 0.1 */
    int32_t flow_blocks;      /* 1..4 */
    int32_t flow_hidden;      /* multiple of 16, <= 256 */
    int32_t train_steps;      /* Adam steps per round */
    int32_t train_batch;      /* rows per step (>= 16) */
    float train_lr;
    uint64_t seed;
    uint64_t capacity;        /* accepted samples kept per round: >= sims_per_round, so no round is truncated */
    abc_mode mode;
    double defensive;         /* prior fraction of a flow round's proposals, in [0, 1) (e.g. 0.1) */
    double val_fraction;      /* held-out fraction for early stopping of the training, in [0, 0.5] (e.g. 0.1) */
    double train_weight_power;/* training weights are (prior / q)^power, in (0, 1] (1: the importance weights;
                                 below 1 the flow fits a broader density between proposal and target) */
    int32_t fresh_init;       /* 1: re-initialise the flow (random, fresh seed) before each training; 0: continue */
    double proposal_scale;    /* base scale tau of the flow proposals (abc_maf_set_proposal_scale), in [0.5, 4]:
                                 1 samples the trained flow; above 1 a broader proposal with heavier coverage
                                 of the tails, weighted by its own density */
    int32_t fallback_rule;    /* ABC_FALLBACK_EFFICIENCY (0) or ABC_FALLBACK_ESS (1), see below */
} abc_smc_config;

/* When a round sends the next one back to the prior (fewer than 64 accepts
 * always does). ABC_FALLBACK_EFFICIENCY: a flow round with defensive draws
 * keeps the flow while ESS / sims_per_round reaches the prior's acceptance
 * rate measured on those draws; a prior round, or a flow round without
 * defensive draws, uses the flow next when its ESS fraction reaches ess_min.
 * ABC_FALLBACK_ESS: every round uses the flow next when its ESS fraction
 * ESS / n_accepted reaches ess_min, and the prior otherwise. */
enum { ABC_FALLBACK_EFFICIENCY = 0, ABC_FALLBACK_ESS = 1 };

typedef struct {
    double eps;
    int32_t proposal;         /* 0 = prior, 1 = flow */
    uint64_t n_sims;
    uint64_t n_accepted;
    uint64_t simulated_days;
    double ess_fraction;      /* ESS / n_accepted of this round's weights */
    float train_loss;         /* flow loss after training on this round (0 if not trained) */
    float ms_propose, ms_simulate, ms_train;
    uint64_t n_defensive;     /* a flow round's proposals drawn from the prior (0 in a prior round) */
    uint64_t n_defensive_accepted; /* how many of them were accepted */
} abc_smc_round;

/* Run cfg->rounds rounds on one region (observed HOST [3][T+1], population
 * N_pop). rounds_out (HOST [cfg->rounds]) receives per-round statistics. The
 * last round's accepted samples go to theta_out (DEVICE float [capacity][8]),
 * weight_out (DEVICE double [capacity], w = prior / q, normalised to sum 1),
 * dist_out (DEVICE double [capacity]); *n_out (HOST) their number (at most
 * capacity). Synchronizes cuda_stream (a non-default stream is required). */
abc_status abc_smc_run(const abc_prior_box* prior, const int32_t* observed, int32_t T, int64_t N_pop,
                       const abc_smc_config* cfg, abc_smc_round* rounds_out, float* theta_out,
                       double* weight_out, double* dist_out, uint64_t* n_out, void* cuda_stream);

/* Sequential ABC with one learned proposal per region, for many regions at
 * once (a stream of chunks): round r runs every region's sims_per_round
 * proposals in one batched launch (abc_plan_*). Region g's tolerance shrinks
 * geometrically to its own final eps over the first shrink_rounds rounds,
 * eps_{g,r} = eps_g / eps_factor^(shrink_rounds - 1 - r), and stays at eps_g
 * afterwards. Each region has its own flow (one set, abc_maf_create_multi);
 * after every round the flows of all regions whose round was good enough are
 * trained together (abc_maf_train_flows) on that round's weighted accepts, and
 * a region falls back to the prior for its next round by the rule of
 * abc_smc_run (defensive mixture included). Every sample accepted at the
 * region's final eps (all rounds from shrink_rounds - 1 on) is pooled in the
 * region's output buffers. Its weight is its round's self-normalised
 * importance weight (prior / q_mix) times the round's effective sample size,
 * so each round's estimate counts in proportion to its ESS; the weighted pool
 * estimates the ABC posterior at eps_g (Eq. 7). From the first round at the
 * final eps on, each region's flow trains on (up to capacity points of) the
 * whole pool instead of the last round alone. Region g simulates with (seed, stream g, index r *
 * sims_per_round + j) and its flow draws with (seed, stream n_regions + g,
 * the same index). The first training of the flows runs base.train_steps
 * Adam steps, later ones (warm starts) train_steps_warm. */
typedef struct {
    const int32_t* observed;  /* HOST int32 [3][T+1] */
    int32_t T;
    int64_t N_pop;
    double eps;               /* the region's final tolerance */
    float* theta_out;         /* DEVICE float [capacity][8]: pooled samples at eps */
    double* weight_out;       /* DEVICE double [capacity]: their weights (ESS-combined across rounds) */
    double* dist_out;         /* DEVICE double [capacity] */
    uint64_t capacity;
    uint64_t n_pooled;        /* out: accepted at eps over all rounds (may exceed capacity) */
    uint64_t n_out;           /* out: samples written, min(n_pooled, capacity) */
} abc_smc_region;

typedef struct {
    abc_smc_config base;      /* rounds, sims_per_round (per region), eps_factor, ess_min, flow shape and
                                 training, seed, capacity (per round and region, >= sims_per_round), mode,
                                 defensive, val_fraction; eps0 unused */
    int32_t shrink_rounds;    /* 1..rounds */
    int32_t train_steps_warm; /* Adam steps of every later training */
} abc_smc_stream_config;

/* rounds_out HOST [rounds][n_regions]. n_regions in 1..ABC_MAX_REGIONS.
 * Synchronizes cuda_stream (non-default). */
abc_status abc_smc_run_regions(const abc_prior_box* prior, abc_smc_region* regions, int32_t n_regions,
                               const abc_smc_stream_config* cfg, abc_smc_round* rounds_out, void* cuda_stream);

/* Plain sequential ABC: population Monte Carlo ABC (Beaumont, Cornuet, Marin,
 * Robert 2009), the SMC-ABC the paper names in Sec. 2.2. Round 0 is rejection
 * from the prior at eps0; round t (eps_t = eps0 * eps_factor^t) proposes
 * theta = theta_j + L z, parent j drawn with probability proportional to its
 * weight, z ~ N(0, I), L L^T = 2 Cov_w(previous population); proposals
 * outside the prior box are not simulated; an accepted particle gets the
 * weight 1 / sum_j w_j exp(-|L^-1 (theta - theta_j)|^2 / 2) (prior over the
 * Gaussian mixture, constants cancelling), normalised to sum 1. Each round
 * simulates batches of `batch` proposals until it holds at least
 * n_particles accepted ones (at most max_batches); all accepted ones of those
 * batches form the population, in ascending sample index (so a seed fixes
 * the whole run, outputs included, while no round accepts more than
 * capacity; beyond it, which samples a round keeps depends on the accept
 * order). Simulations use (seed, stream 0, index), proposals (seed, stream 2,
 * index). theta_out (float [n][8]), weight_out and dist_out (double [n]) may
 * be host or device memory; *n_out = n, the final population's size. */
typedef struct {
    int32_t rounds;
    uint64_t n_particles;
    uint64_t batch;
    int32_t max_batches;
    double eps0;
    double eps_factor;
    uint64_t seed;
    uint64_t capacity;        /* population buffer size (>= n_particles) */
    abc_mode mode;
} abc_pmc_config;

typedef struct {
    double eps;
    uint64_t n_sims;          /* proposals generated */
    uint64_t n_accepted;      /* population size */
    double ess_fraction;
    float ms;
} abc_pmc_round;

abc_status abc_pmc_run(const abc_prior_box* prior, const int32_t* observed, int32_t T, int64_t N_pop,
                       const abc_pmc_config* cfg, abc_pmc_round* rounds_out, float* theta_out,
                       double* weight_out, double* dist_out, uint64_t* n_out, void* cuda_stream);

/* The population Monte Carlo pieces on their own, for tests and custom loops:
 * proposals (DEVICE float [n][8], NaN first coordinate = outside the box) from
 * a weighted population (DEVICE float [m][8], DEVICE double weights [m]) and
 * the lower-triangular L (HOST float [8][8], row-major); and the weights of
 * new particles (DEVICE float [n][8] -> DEVICE double [n]) against the old
 * population. Async on cuda_stream. */
abc_status abc_pmc_propose(const abc_prior_box* prior, const float* theta_old, const double* w_old, uint64_t m,
                           const float* L, uint64_t seed, uint64_t first_index, uint64_t n, float* theta_out,
                           void* cuda_stream);
abc_status abc_pmc_weights(const float* theta_new, uint64_t n, const float* theta_old, const double* w_old,
                           uint64_t m, const float* L, double* w_out, void* cuda_stream);

/* Variant of abc_sample that allocates no memory. It is for callers that must
 * not allocate device memory while sampling: code running inside a host
 * framework that owns the GPU's memory pool and forbids other allocators, or
 * services that allocate everything once at start-up and must not allocate
 * (or risk an out-of-memory failure) in their steady state. It has no
 * counterpart in the paper; it only changes where the scratch memory comes from.
 *
 * Arguments, outputs, errors and results are those of abc_sample (the same
 * kernel runs), for T <= ABC_NOALLOC_T_MAX; a larger T returns
 * ABC_ERR_INVALID_ARG. The scratch (three counters and the observed series) is
 * a fixed ABC_NOALLOC_SCRATCH_BYTES array of device memory declared at file
 * scope in this library, so every GPU that loads the library holds it until the
 * process exits. The first call on each device looks up that array's device
 * address with the device current (a one-time set-up done by that call); make
 * the first call on a device before any stream capture. If that lookup fails,
 * the call returns ABC_ERR_CUDA and the next call on the device tries again. All calls share the one
 * array and each call zeroes the counters it uses: calls that overlap on the GPU
 * (different streams or host threads) race on it and must be serialized by the
 * caller. Calls no cudaMalloc, cudaMallocAsync or cudaFree. */
#define ABC_NOALLOC_T_MAX 1024
#define ABC_NOALLOC_SCRATCH_BYTES (256 + 16 * (ABC_NOALLOC_T_MAX + 1))
abc_status abc_sample_noalloc(const abc_prior_box* prior, const int32_t* observed, int32_t T,
                              int64_t N_pop, double eps, uint64_t n_samples, uint64_t seed,
                              uint32_t stream, abc_mode mode, uint64_t first_index,
                              float* theta_out, double* dist_out, uint64_t* idx_out,
                              uint64_t capacity, uint64_t* n_accepted, void* cuda_stream);

/* Number of model days simulated by the last successful abc_sample call on
 * this thread. abc_sample stops simulating a sample once its running distance^2
 * exceeds eps^2 (the partial sums only grow, so it could not be accepted); the
 * accept set is the same as simulating all T days of every sample. This count is
 * the work actually done: at most n_samples * T. */
uint64_t abc_last_simulated_days(void);

/* Static description of a status code. */
const char* abc_strerror(abc_status status);

/* Thread-local detail of the last error returned on this thread ("" if none). */
const char* abc_last_error(void);

/* Library version: major * 10000 + minor * 100 + patch. */
int abc_version(void);

#ifdef __cplusplus
}
#endif
#endif /* ABC_GB300_H */
