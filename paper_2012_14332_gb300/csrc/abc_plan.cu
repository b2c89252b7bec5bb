// abc_plan.cu -- the batched-regions ABI (abc_plan_*): plan creation with all
// device memory allocated up front, allocation-free asynchronous runs, CUDA
// graph capture and replay of runs, and the launch-shape autotuner.
#include <cmath>
#include <cstddef>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/abc_gb300.h"
#include "abc_kernels.h"
#include "abc_model.cuh"

namespace abcgb {
// shared with abc_api.cu
abc_status plan_fail(abc_status st, const char* msg);
abc_status plan_cuda_fail(cudaError_t e, const char* what);
abc_status plan_ok();
bool plan_check_prior(const abc_prior_box* prior, abc_status* st);
uint64_t plan_acc_threshold(double eps);
ModelParams plan_make_params(const abc_prior_box* prior, int32_t T, int64_t N_pop, uint64_t seed, uint32_t stream,
                             const int32_t* ard0);
}  // namespace abcgb

struct abc_plan_s {
    int device = 0;
    bool fast = true;
    abcgb::ModelParams p{};
    int32_t n_regions = 0;
    std::vector<abcgb::RegionDev> regions;   // host copy of the table
    abcgb::RegionDev* d_regions = nullptr;
    int4* d_obs = nullptr;
    unsigned long long* d_next = nullptr;
    unsigned long long* d_counters = nullptr;
    float* d_theta = nullptr;
    double* d_dist = nullptr;
    uint64_t* d_idx = nullptr;
    uint64_t total_chunks = 0;
    int32_t n_obs_smem = 0;   // observed days staged in shared memory by the kernel (0: read through the cache)
    abcgb::BatchShape shape{256, 1, 0, 0};
    cudaGraphExec_t graph = nullptr;
    int32_t graph_runs = 0;
    bool graph_below62 = false;   // the kernel variant the graph was captured with
};

namespace {

using abcgb::plan_cuda_fail;
using abcgb::plan_fail;
using abcgb::plan_ok;

#define PLAN_TRY(expr, what)                                  \
    do {                                                      \
        cudaError_t _e = (expr);                              \
        if (_e != cudaSuccess) return plan_cuda_fail(_e, what); \
    } while (0)

abc_status check_plan(abc_plan plan)
{
    if (!plan) return plan_fail(ABC_ERR_INVALID_ARG, "plan is NULL");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != plan->device)
        return plan_fail(ABC_ERR_INVALID_ARG, "the plan's device is not the current device");
    return ABC_OK;
}

void free_plan(abc_plan_s* pl)
{
    if (pl->graph) cudaGraphExecDestroy(pl->graph);
    cudaFree(pl->d_regions);
    cudaFree(pl->d_obs);
    cudaFree(pl->d_next);
    cudaFree(pl->d_counters);
    cudaFree(pl->d_theta);
    cudaFree(pl->d_dist);
    cudaFree(pl->d_idx);
    delete pl;
}

abc_status upload_table(abc_plan plan)
{
    PLAN_TRY(cudaMemcpy(plan->d_regions, plan->regions.data(), sizeof(abcgb::RegionDev) * plan->n_regions,
                        cudaMemcpyHostToDevice),
             "cudaMemcpy(region table)");
    return ABC_OK;
}

// every region's threshold below 2^62: the batched kernel's cheaper variant
bool below62(const abc_plan_s* plan)
{
    for (int32_t r = 0; r < plan->n_regions; ++r)
        if (plan->regions[r].acc_max >= 0x4000000000000000ull) return false;
    return true;
}

abc_status run_once(abc_plan plan, cudaStream_t s)
{
    PLAN_TRY(cudaMemsetAsync(plan->d_next, 0, sizeof(unsigned long long), s), "cudaMemsetAsync(claims)");
    abcgb::BatchArgs a;
    a.regions = plan->d_regions;
    a.n_regions = plan->n_regions;
    a.total_chunks = plan->total_chunks;
    a.obs = plan->d_obs;
    a.n_obs_smem = plan->n_obs_smem;
    a.next = plan->d_next;
    PLAN_TRY(abcgb::launch_batch(plan->p, a, plan->fast, below62(plan), plan->shape, s), "abc_batch_kernel launch");
    PLAN_TRY(abcgb::launch_advance(plan->d_regions, plan->n_regions, s), "advance launch");
    return ABC_OK;
}

}  // namespace

extern "C" {

abc_status abc_plan_create(const abc_prior_box* prior, const abc_region* regions, int32_t n_regions, uint64_t seed,
                           abc_mode mode, abc_plan* plan_out)
{
    abc_status st = ABC_OK;
    if (!plan_out) return plan_fail(ABC_ERR_INVALID_ARG, "plan_out is NULL");
    *plan_out = nullptr;
    if (!abcgb::plan_check_prior(prior, &st)) return st;
    if (!regions || n_regions < 1 || n_regions > ABC_MAX_REGIONS)
        return plan_fail(ABC_ERR_INVALID_ARG, "n_regions must be in [1, ABC_MAX_REGIONS] with a region array");
    if (mode != ABC_EXACT && mode != ABC_FAST) return plan_fail(ABC_ERR_INVALID_ARG, "unknown mode");
    std::vector<int4> obs;
    std::vector<abcgb::RegionDev> table(n_regions);
    uint64_t chunks = 0, cap_total = 0;
    for (int32_t r = 0; r < n_regions; ++r) {
        const abc_region& g = regions[r];
        char msg[160];
        if (g.T < 1 || g.T > ABC_T_MAX) {
            snprintf(msg, sizeof msg, "region %d: T = %d outside [1, %d]", r, g.T, ABC_T_MAX);
            return plan_fail(ABC_ERR_INVALID_ARG, msg);
        }
        if (g.N_pop < 1 || g.N_pop >= ((int64_t)1 << 31)) {
            snprintf(msg, sizeof msg, "region %d: N_pop outside [1, 2^31)", r);
            return plan_fail(ABC_ERR_INVALID_ARG, msg);
        }
        if (!(g.eps >= 0.0)) {
            snprintf(msg, sizeof msg, "region %d: eps must be >= 0 and not NaN", r);
            return plan_fail(ABC_ERR_INVALID_ARG, msg);
        }
        if (g.stream > ABC_STREAM_MAX || !g.observed) {
            snprintf(msg, sizeof msg, "region %d: stream above 2^30 - 1 or observed is NULL", r);
            return plan_fail(ABC_ERR_INVALID_ARG, msg);
        }
        abcgb::RegionDev& R = table[r];
        std::memset(&R, 0, sizeof R);
        R.obs_off = (uint32_t)obs.size();
        for (int32_t d = 0; d <= g.T; ++d) {
            const int32_t A = g.observed[d], Rr = g.observed[(g.T + 1) + d], D = g.observed[2 * (g.T + 1) + d];
            if (A < 0 || Rr < 0 || D < 0) {
                snprintf(msg, sizeof msg, "region %d: negative observed count on day %d", r, d);
                return plan_fail(ABC_ERR_INVALID_ARG, msg);
            }
            obs.push_back(make_int4(A, Rr, D, 0));
        }
        const int4 o0 = obs[R.obs_off];
        if ((int64_t)o0.x + o0.y + o0.z > g.N_pop) {
            snprintf(msg, sizeof msg, "region %d: A0 + R0 + D0 exceeds N_pop", r);
            return plan_fail(ABC_ERR_INVALID_ARG, msg);
        }
        const int32_t ard0[3] = {o0.x, o0.y, o0.z};
        const abcgb::ModelParams rp = abcgb::plan_make_params(prior, g.T, g.N_pop, seed, g.stream, ard0);
        R.first_index = g.first_index;
        R.n_samples = g.n_samples;
        R.chunk_begin = chunks;
        R.acc_max = abcgb::plan_acc_threshold(g.eps);
        R.capacity = g.capacity;
        R.theta_in = g.theta_in;
        R.T = g.T;
        R.P = rp.P;
        R.room0 = rp.room0;
        R.A0 = rp.A0;
        R.R0 = rp.R0;
        R.D0 = rp.D0;
        R.ctr3_base = rp.ctr3_base;
        R.inv_p = rp.inv_p;
        chunks += (g.n_samples + 31) / 32;
        cap_total += g.capacity;
    }
    abc_plan_s* pl = new abc_plan_s();
    PLAN_TRY(cudaGetDevice(&pl->device), "cudaGetDevice");
    pl->fast = mode == ABC_FAST;
    // until tuned: in fast mode the shape the autotuner chose on the three-
    // and sixteen-region workloads (the lean form, two day pairs per
    // iteration); the standard one-pair form in exact mode
    if (pl->fast) pl->shape = abcgb::BatchShape{256, 2, 0, 1};
    pl->p = abcgb::plan_make_params(prior, 1, 1, seed, 0, nullptr);
    pl->n_regions = n_regions;
    pl->total_chunks = chunks;
    auto cleanup = [pl](abc_status e) {
        free_plan(pl);
        return e;
    };
    cudaError_t e;
    if ((e = cudaMalloc(&pl->d_regions, sizeof(abcgb::RegionDev) * n_regions)) != cudaSuccess ||
        (e = cudaMalloc(&pl->d_obs, sizeof(int4) * obs.size())) != cudaSuccess ||
        (e = cudaMalloc(&pl->d_next, sizeof(unsigned long long))) != cudaSuccess ||
        (e = cudaMalloc(&pl->d_counters, 2 * sizeof(unsigned long long) * n_regions)) != cudaSuccess ||
        (e = cudaMalloc(&pl->d_theta, sizeof(float) * 8 * (cap_total ? cap_total : 1))) != cudaSuccess ||
        (e = cudaMalloc(&pl->d_dist, sizeof(double) * (cap_total ? cap_total : 1))) != cudaSuccess ||
        (e = cudaMalloc(&pl->d_idx, sizeof(uint64_t) * (cap_total ? cap_total : 1))) != cudaSuccess)
        return cleanup(plan_cuda_fail(e, "cudaMalloc(plan)"));
    uint64_t off = 0;
    for (int32_t r = 0; r < n_regions; ++r) {
        table[r].theta_out = pl->d_theta + 8 * off;
        table[r].dist_out = pl->d_dist + off;
        table[r].idx_out = pl->d_idx + off;
        table[r].counters = pl->d_counters + 2 * r;
        off += table[r].capacity;
    }
    pl->regions = table;
    if ((e = cudaMemcpy(pl->d_obs, obs.data(), sizeof(int4) * obs.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(pl->d_counters, 0, 2 * sizeof(unsigned long long) * n_regions)) != cudaSuccess)
        return cleanup(plan_cuda_fail(e, "plan upload"));
    if ((st = upload_table(pl)) != ABC_OK) return cleanup(st);
    // both distance-accumulation variants: either may be launched (or captured) later
    // several regions' series in shared memory: measured 1.5-2 % faster on 3 and 16
    // regions; one region's series is read through the cache (0.5 % faster there)
    pl->n_obs_smem = n_regions > 1 && obs.size() <= (size_t)abcgb::kBatchObsSmemMax ? (int32_t)obs.size() : 0;
    if ((e = abcgb::prepare_batch(pl->fast, true, pl->n_obs_smem, pl->shape)) != cudaSuccess ||
        (e = abcgb::prepare_batch(pl->fast, false, pl->n_obs_smem, pl->shape)) != cudaSuccess)
        return cleanup(plan_cuda_fail(e, "prepare_batch"));
    *plan_out = pl;
    return plan_ok();
}

abc_status abc_plan_reset(abc_plan plan, void* cuda_stream)
{
    abc_status st;
    if ((st = check_plan(plan)) != ABC_OK) return st;
    PLAN_TRY(cudaMemsetAsync(plan->d_counters, 0, 2 * sizeof(unsigned long long) * plan->n_regions,
                             (cudaStream_t)cuda_stream),
             "cudaMemsetAsync(counters)");
    return plan_ok();
}

abc_status abc_plan_run(abc_plan plan, void* cuda_stream)
{
    abc_status st;
    if ((st = check_plan(plan)) != ABC_OK) return st;
    if ((st = run_once(plan, (cudaStream_t)cuda_stream)) != ABC_OK) return st;
    return plan_ok();
}

abc_status abc_plan_run_graph(abc_plan plan, int32_t n_runs, void* cuda_stream)
{
    abc_status st;
    if ((st = check_plan(plan)) != ABC_OK) return st;
    if (n_runs < 1) return plan_fail(ABC_ERR_INVALID_ARG, "n_runs must be >= 1");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (!plan->graph || plan->graph_runs != n_runs || plan->graph_below62 != below62(plan)) {
        if (!s) return plan_fail(ABC_ERR_INVALID_ARG, "graph capture needs a non-default stream");
        if (plan->graph) {
            cudaGraphExecDestroy(plan->graph);
            plan->graph = nullptr;
        }
        cudaGraph_t g = nullptr;
        PLAN_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
        for (int32_t r = 0; r < n_runs; ++r) {
            if ((st = run_once(plan, s)) != ABC_OK) {
                cudaStreamEndCapture(s, &g);
                if (g) cudaGraphDestroy(g);
                return st;
            }
        }
        PLAN_TRY(cudaStreamEndCapture(s, &g), "cudaStreamEndCapture");
        cudaError_t e = cudaGraphInstantiate(&plan->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            plan->graph = nullptr;
            return plan_cuda_fail(e, "cudaGraphInstantiate");
        }
        plan->graph_runs = n_runs;
        plan->graph_below62 = below62(plan);
    }
    PLAN_TRY(cudaGraphLaunch(plan->graph, s), "cudaGraphLaunch");
    return plan_ok();
}

abc_status abc_plan_tune(abc_plan plan, void* cuda_stream, abc_launch_shape* shapes_out, int32_t max_shapes,
                         int32_t* n_shapes_out, abc_launch_shape* best_out)
{
    abc_status st;
    if ((st = check_plan(plan)) != ABC_OK) return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // the tuning runs consume sample ranges and add to the counters: save both
    PLAN_TRY(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    std::vector<abcgb::RegionDev> saved(plan->n_regions);
    std::vector<unsigned long long> saved_counters(2 * plan->n_regions);
    PLAN_TRY(cudaMemcpy(saved.data(), plan->d_regions, sizeof(abcgb::RegionDev) * plan->n_regions,
                        cudaMemcpyDeviceToHost),
             "cudaMemcpy(region table)");
    PLAN_TRY(cudaMemcpy(saved_counters.data(), plan->d_counters, sizeof(unsigned long long) * saved_counters.size(),
                        cudaMemcpyDeviceToHost),
             "cudaMemcpy(counters)");
    cudaEvent_t e0, e1;
    PLAN_TRY(cudaEventCreate(&e0), "cudaEventCreate");
    PLAN_TRY(cudaEventCreate(&e1), "cudaEventCreate");
    const abcgb::BatchShape keep = plan->shape;
    int best = -1;
    float best_ms = 0.0f;
    const int n = abcgb::batch_shape_count();
    int written = 0;
    abc_status result = ABC_OK;
    for (int c = 0; c < n && result == ABC_OK; ++c) {
        if (!abcgb::batch_shape_supported(abcgb::batch_shape(c), plan->fast)) continue;
        plan->shape = abcgb::batch_shape(c);
        // both distance variants: a later abc_plan_set_eps may switch to the other
        cudaError_t e = abcgb::prepare_batch(plan->fast, true, plan->n_obs_smem, plan->shape);
        if (e == cudaSuccess) e = abcgb::prepare_batch(plan->fast, false, plan->n_obs_smem, plan->shape);
        if (e != cudaSuccess) { result = plan_cuda_fail(e, "prepare_batch"); break; }
        float ms = 0.0f;
        // one untimed run to warm up, one timed run; both on tuning sample ranges
        for (int rep = 0; rep < 2 && result == ABC_OK; ++rep) {
            if (cudaEventRecord(e0, s) != cudaSuccess) { result = plan_fail(ABC_ERR_CUDA, "cudaEventRecord"); break; }
            if ((result = run_once(plan, s)) != ABC_OK) break;
            if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
                result = plan_fail(ABC_ERR_CUDA, "timing a tuning run");
        }
        if (result != ABC_OK) break;
        if (shapes_out && written < max_shapes) {
            shapes_out[written] = abc_launch_shape{plan->shape.block_threads, plan->shape.pairs,
                                                   plan->shape.blocks_per_sm, plan->shape.lean, ms};
            ++written;
        }
        if (best < 0 || ms < best_ms) {
            best = c;
            best_ms = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    plan->shape = best >= 0 ? abcgb::batch_shape(best) : keep;
    cudaStreamSynchronize(s);
    // put the sample ranges and counters back as they were before tuning
    PLAN_TRY(cudaMemcpy(plan->d_regions, saved.data(), sizeof(abcgb::RegionDev) * plan->n_regions,
                        cudaMemcpyHostToDevice),
             "cudaMemcpy(region table)");
    PLAN_TRY(cudaMemcpy(plan->d_counters, saved_counters.data(), sizeof(unsigned long long) * saved_counters.size(),
                        cudaMemcpyHostToDevice),
             "cudaMemcpy(counters)");
    if (result != ABC_OK) return result;
    if (plan->graph) {
        cudaGraphExecDestroy(plan->graph);
        plan->graph = nullptr;
    }
    if (n_shapes_out) *n_shapes_out = written;
    if (best_out)
        *best_out = abc_launch_shape{plan->shape.block_threads, plan->shape.pairs, plan->shape.blocks_per_sm,
                                     plan->shape.lean, best_ms};
    return plan_ok();
}

abc_status abc_plan_results(abc_plan plan, int32_t region, uint64_t* n_accepted, uint64_t* simulated_days,
                            float** theta_out, double** dist_out, uint64_t** idx_out, void* cuda_stream)
{
    abc_status st;
    if ((st = check_plan(plan)) != ABC_OK) return st;
    if (region < 0 || region >= plan->n_regions) return plan_fail(ABC_ERR_INVALID_ARG, "region out of range");
    unsigned long long c[2] = {0, 0};
    cudaStream_t s = (cudaStream_t)cuda_stream;
    PLAN_TRY(cudaMemcpyAsync(c, plan->d_counters + 2 * region, sizeof c, cudaMemcpyDeviceToHost, s),
             "cudaMemcpyAsync(counters)");
    PLAN_TRY(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    const abcgb::RegionDev& R = plan->regions[region];
    if (n_accepted) *n_accepted = c[0];
    if (simulated_days) *simulated_days = c[1];
    if (theta_out) *theta_out = R.theta_out;
    if (dist_out) *dist_out = R.dist_out;
    if (idx_out) *idx_out = R.idx_out;
    return plan_ok();
}

abc_status abc_plan_copy_results(abc_plan plan, int32_t region, float* theta_dst, double* dist_dst,
                                 uint64_t* idx_dst, uint64_t count, uint64_t* copied, void* cuda_stream)
{
    uint64_t n = 0;
    abc_status st = abc_plan_results(plan, region, &n, nullptr, nullptr, nullptr, nullptr, cuda_stream);
    if (st != ABC_OK) return st;
    const abcgb::RegionDev& R = plan->regions[region];
    if (n > R.capacity) n = R.capacity;
    if (n > count) n = count;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (n > 0) {
        if (theta_dst)
            PLAN_TRY(cudaMemcpyAsync(theta_dst, R.theta_out, sizeof(float) * 8 * n, cudaMemcpyDefault, s),
                     "cudaMemcpyAsync(theta)");
        if (dist_dst)
            PLAN_TRY(cudaMemcpyAsync(dist_dst, R.dist_out, sizeof(double) * n, cudaMemcpyDefault, s),
                     "cudaMemcpyAsync(dist)");
        if (idx_dst)
            PLAN_TRY(cudaMemcpyAsync(idx_dst, R.idx_out, sizeof(uint64_t) * n, cudaMemcpyDefault, s),
                     "cudaMemcpyAsync(idx)");
    }
    if (copied) *copied = n;
    return plan_ok();
}

abc_status abc_plan_set_region(abc_plan plan, int32_t region, const float* theta_in, uint64_t first_index)
{
    abc_status st;
    if ((st = check_plan(plan)) != ABC_OK) return st;
    if (region < 0 || region >= plan->n_regions) return plan_fail(ABC_ERR_INVALID_ARG, "region out of range");
    // keep the device table's current first indices of the other regions
    std::vector<abcgb::RegionDev> cur(plan->n_regions);
    PLAN_TRY(cudaMemcpy(cur.data(), plan->d_regions, sizeof(abcgb::RegionDev) * plan->n_regions,
                        cudaMemcpyDeviceToHost),
             "cudaMemcpy(region table)");
    cur[region].theta_in = theta_in;
    cur[region].first_index = first_index;
    plan->regions[region].theta_in = theta_in;
    plan->regions[region].first_index = first_index;
    PLAN_TRY(cudaMemcpy(plan->d_regions, cur.data(), sizeof(abcgb::RegionDev) * plan->n_regions,
                        cudaMemcpyHostToDevice),
             "cudaMemcpy(region table)");
    return plan_ok();
}

abc_status abc_plan_set_shape(abc_plan plan, const abc_launch_shape* shape)
{
    abc_status st;
    if ((st = check_plan(plan)) != ABC_OK) return st;
    if (!shape) return plan_fail(ABC_ERR_INVALID_ARG, "shape is NULL");
    for (int c = 0; c < abcgb::batch_shape_count(); ++c) {
        const abcgb::BatchShape b = abcgb::batch_shape(c);
        if (b.block_threads != shape->block_threads || b.pairs != shape->pairs_per_iteration ||
            b.blocks_per_sm != shape->blocks_per_sm || b.lean != shape->lean)
            continue;
        if (!abcgb::batch_shape_supported(b, plan->fast))
            return plan_fail(ABC_ERR_INVALID_ARG, "the lean kernel form is compiled for fast mode only");
        PLAN_TRY(abcgb::prepare_batch(plan->fast, true, plan->n_obs_smem, b), "prepare_batch");
        PLAN_TRY(abcgb::prepare_batch(plan->fast, false, plan->n_obs_smem, b), "prepare_batch");
        plan->shape = b;
        if (plan->graph) {
            cudaGraphExecDestroy(plan->graph);
            plan->graph = nullptr;
        }
        return plan_ok();
    }
    return plan_fail(ABC_ERR_INVALID_ARG, "the library is not compiled for this launch shape");
}

abc_status abc_plan_set_eps(abc_plan plan, int32_t region, double eps)
{
    abc_status st;
    if ((st = check_plan(plan)) != ABC_OK) return st;
    if (region < 0 || region >= plan->n_regions) return plan_fail(ABC_ERR_INVALID_ARG, "region out of range");
    if (!(eps >= 0.0)) return plan_fail(ABC_ERR_INVALID_ARG, "eps must be >= 0 and not NaN");
    const uint64_t acc_max = abcgb::plan_acc_threshold(eps);
    plan->regions[region].acc_max = acc_max;
    // one field of the device table; the rest (first indices advanced by runs) stays
    abcgb::RegionDev* d = plan->d_regions + region;
    PLAN_TRY(cudaMemcpy(reinterpret_cast<char*>(d) + offsetof(abcgb::RegionDev, acc_max), &acc_max, sizeof acc_max,
                        cudaMemcpyHostToDevice),
             "cudaMemcpy(region eps)");
    return plan_ok();
}

abc_status abc_plan_destroy(abc_plan plan)
{
    if (!plan) return plan_fail(ABC_ERR_INVALID_ARG, "plan is NULL");
    free_plan(plan);
    // leaves the thread's last error as it was: drivers destroy their plans on
    // the way out of a failed call
    return ABC_OK;
}

}  // extern "C"

namespace abcgb {

// Every region's results of the last run at once: what abc_plan_results gives
// for each region, read with one copy and one synchronisation of s. The
// arrays hold n_regions entries each.
abc_status plan_results_all(abc_plan plan, uint64_t* n_accepted, uint64_t* simulated_days, float** theta_out,
                            double** dist_out, uint64_t** idx_out, void* cuda_stream)
{
    abc_status st;
    if ((st = check_plan(plan)) != ABC_OK) return st;
    const int32_t R = plan->n_regions;
    std::vector<unsigned long long> c(2 * (size_t)R);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    PLAN_TRY(cudaMemcpyAsync(c.data(), plan->d_counters, sizeof(unsigned long long) * c.size(), cudaMemcpyDeviceToHost,
                             s),
             "cudaMemcpyAsync(counters)");
    PLAN_TRY(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    for (int32_t g = 0; g < R; ++g) {
        const abcgb::RegionDev& Rg = plan->regions[g];
        n_accepted[g] = c[2 * (size_t)g];
        simulated_days[g] = c[2 * (size_t)g + 1];
        theta_out[g] = Rg.theta_out;
        dist_out[g] = Rg.dist_out;
        idx_out[g] = Rg.idx_out;
    }
    return plan_ok();
}

}  // namespace abcgb
