// abc_smc.cu -- sequential ABC with the learned flow proposal: the host loop
// over rounds (propose, simulate and accept, weight, train, shrink eps).
// Every step runs in the library's kernels: the flow sampler and trainer
// (abc_maf.cu) and the batched rejection kernel of a one-region plan
// (abc_batch.cu) reading the proposals from device memory.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/abc_gb300.h"
#include "abc_model.cuh"

namespace abcgb {
abc_status plan_fail(abc_status st, const char* msg);
abc_status plan_cuda_fail(cudaError_t e, const char* what);
abc_status plan_ok();
bool plan_check_prior(const abc_prior_box* prior, abc_status* st);
ModelParams plan_make_params(const abc_prior_box* prior, int32_t T, int64_t N_pop, uint64_t seed, uint32_t stream,
                             const int32_t* ard0);
}  // namespace abcgb

namespace {

// log q of each accepted sample, looked up by its index in the round's proposals.
__global__ void gather_logq_kernel(const float* __restrict__ logq, const uint64_t* __restrict__ idx, uint64_t first,
                                   uint64_t n, float* __restrict__ out)
{
    const uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) out[j] = logq[idx[j] - first];
}

// prior draws of sample indices first .. first + n - 1 (stream 0, the words the
// plain sampler would use for those indices)
__global__ void prior_theta_kernel(const __grid_constant__ abcgb::ModelParams p, uint64_t first, uint64_t n,
                                   float* __restrict__ theta)
{
    const uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    float th[8];
    abcgb::prior_draw(p, first + j, th);
    float4* o = reinterpret_cast<float4*>(theta + 8 * j);
    o[0] = make_float4(th[0], th[1], th[2], th[3]);
    o[1] = make_float4(th[4], th[5], th[6], th[7]);
}

// log q_mix = log((1 - lam) q + lam prior), in place over log q
__global__ void mixture_logq_kernel(float* __restrict__ logq, uint64_t n, float log_1m_lam, float log_lam_prior)
{
    const uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const float a = log_1m_lam + logq[j], b = log_lam_prior;
    const float m = fmaxf(a, b);
    logq[j] = m + log1pf(expf(-fabsf(a - b)));
}

struct Guard {
    std::vector<void*> dev;
    abc_plan plan = nullptr;
    abc_maf flow = nullptr;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    ~Guard()
    {
        for (void* p : dev) cudaFree(p);
        if (plan) abc_plan_destroy(plan);
        if (flow) abc_maf_destroy(flow);
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
    }
};

}  // namespace

using abcgb::plan_cuda_fail;
using abcgb::plan_fail;

#define SMC_TRY(expr, what)                                   \
    do {                                                      \
        cudaError_t _e = (expr);                              \
        if (_e != cudaSuccess) return plan_cuda_fail(_e, what); \
    } while (0)
#define SMC_ST(expr)                        \
    do {                                    \
        abc_status _s = (expr);             \
        if (_s != ABC_OK) return _s;        \
    } while (0)

extern "C" abc_status abc_smc_run(const abc_prior_box* prior, const int32_t* observed, int32_t T, int64_t N_pop,
                                  const abc_smc_config* cfg, abc_smc_round* rounds_out, float* theta_out,
                                  double* weight_out, double* dist_out, uint64_t* n_out, void* cuda_stream)
{
    abc_status st;
    if (!abcgb::plan_check_prior(prior, &st)) return st;
    if (!cfg || !rounds_out || !n_out) return plan_fail(ABC_ERR_INVALID_ARG, "cfg, rounds_out and n_out are required");
    if (cfg->rounds < 1 || cfg->sims_per_round == 0 || !(cfg->eps0 >= 0.0) || !(cfg->eps_factor > 0.0) ||
        cfg->eps_factor > 1.0 || !(cfg->ess_min >= 0.0) || cfg->capacity == 0 || !(cfg->defensive >= 0.0) ||
        cfg->defensive >= 1.0)
        return plan_fail(ABC_ERR_INVALID_ARG, "bad sequential ABC configuration");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (!s) return plan_fail(ABC_ERR_INVALID_ARG, "sequential ABC needs a non-default stream");
    const uint64_t N = cfg->sims_per_round, cap = cfg->capacity;
    double log_prior = 0.0;
    for (int j = 0; j < 8; ++j) log_prior -= std::log((double)prior->hi[j] - (double)prior->lo[j]);

    Guard gd;
    SMC_ST(abc_maf_create(cfg->flow_blocks, cfg->flow_hidden, prior, &gd.flow));
    SMC_ST(abc_maf_init_random(gd.flow, cfg->seed ^ 0x5EED5EEDull, 0.3f));
    float *d_prop = nullptr, *d_logq = nullptr, *d_acc_logq = nullptr, *d_w = nullptr;
    SMC_TRY(cudaMalloc(&d_prop, sizeof(float) * 8 * N), "cudaMalloc(proposals)");
    gd.dev.push_back(d_prop);
    SMC_TRY(cudaMalloc(&d_logq, sizeof(float) * N), "cudaMalloc(logq)");
    gd.dev.push_back(d_logq);
    SMC_TRY(cudaMalloc(&d_acc_logq, sizeof(float) * cap), "cudaMalloc(accepted logq)");
    gd.dev.push_back(d_acc_logq);
    SMC_TRY(cudaMalloc(&d_w, sizeof(float) * cap), "cudaMalloc(weights)");
    gd.dev.push_back(d_w);
    float* d_train = nullptr;
    SMC_TRY(cudaMalloc(&d_train, sizeof(float) * 8 * cap), "cudaMalloc(training set)");
    gd.dev.push_back(d_train);
    for (cudaEvent_t& e : gd.ev) SMC_TRY(cudaEventCreate(&e), "cudaEventCreate");

    double eps = cfg->eps0;
    bool use_flow = false;
    std::vector<float> h_logq(cap), h_w(cap);
    std::vector<double> h_wd(cap);
    uint64_t last_n = 0;
    for (int32_t r = 0; r < cfg->rounds; ++r) {
        abc_smc_round& R = rounds_out[r];
        R = abc_smc_round{};
        R.eps = eps;
        R.proposal = use_flow ? 1 : 0;
        R.n_sims = N;
        const uint64_t first = (uint64_t)r * N;
        SMC_TRY(cudaEventRecord(gd.ev[0], s), "cudaEventRecord");
        if (use_flow) {
            // (1 - defensive) N flow draws, the rest prior draws, all weighted by the mixture density
            const uint64_t n_prior = (uint64_t)std::floor(cfg->defensive * (double)N);
            const uint64_t n_flow = N - n_prior;
            // flow draws carry the sampler's log q (exact for the drawn point); the
            // prior draws get the flow's density evaluated at them
            if (n_flow) SMC_ST(abc_maf_sample(gd.flow, n_flow, nullptr, cfg->seed, 1, first, d_prop, d_logq, s));
            if (n_prior) {
                const abcgb::ModelParams pp = abcgb::plan_make_params(prior, 1, 1, cfg->seed, 0, nullptr);
                prior_theta_kernel<<<(unsigned)((n_prior + 255) / 256), 256, 0, s>>>(pp, first + n_flow, n_prior,
                                                                                   d_prop + 8 * n_flow);
                SMC_TRY(cudaGetLastError(), "prior draw launch");
                SMC_ST(abc_maf_log_q(gd.flow, n_prior, d_prop + 8 * n_flow, d_logq + n_flow, s));
            }
            if (cfg->defensive > 0.0) {
                mixture_logq_kernel<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(
                    d_logq, N, (float)std::log1p(-cfg->defensive), (float)(std::log(cfg->defensive) + log_prior));
                SMC_TRY(cudaGetLastError(), "mixture launch");
            }
        }
        SMC_TRY(cudaEventRecord(gd.ev[1], s), "cudaEventRecord");
        abc_region reg{};
        reg.observed = observed;
        reg.T = T;
        reg.N_pop = N_pop;
        reg.eps = eps;
        reg.n_samples = N;
        reg.first_index = first;
        reg.stream = 0;
        reg.capacity = cap;
        reg.theta_in = use_flow ? d_prop : nullptr;
        if (gd.plan) {
            abc_plan_destroy(gd.plan);
            gd.plan = nullptr;
        }
        SMC_ST(abc_plan_create(prior, &reg, 1, cfg->seed, cfg->mode, &gd.plan));
        SMC_ST(abc_plan_run(gd.plan, s));
        SMC_TRY(cudaEventRecord(gd.ev[2], s), "cudaEventRecord");
        uint64_t n_acc = 0, days = 0;
        float* acc_theta = nullptr;
        double* acc_dist = nullptr;
        uint64_t* acc_idx = nullptr;
        SMC_ST(abc_plan_results(gd.plan, 0, &n_acc, &days, &acc_theta, &acc_dist, &acc_idx, s));
        R.n_accepted = n_acc;
        R.simulated_days = days;
        const uint64_t m = std::min(n_acc, cap);
        // importance weights prior / q of the kept accepted samples
        if (m > 0) {
            if (use_flow) {
                gather_logq_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(d_logq, acc_idx, first, m, d_acc_logq);
                SMC_TRY(cudaGetLastError(), "gather launch");
                SMC_TRY(cudaMemcpyAsync(h_logq.data(), d_acc_logq, sizeof(float) * m, cudaMemcpyDeviceToHost, s),
                        "cudaMemcpyAsync(logq)");
                SMC_TRY(cudaStreamSynchronize(s), "cudaStreamSynchronize");
                double top = -INFINITY;
                for (uint64_t j = 0; j < m; ++j) top = std::max(top, log_prior - (double)h_logq[j]);
                for (uint64_t j = 0; j < m; ++j) h_wd[j] = std::exp(log_prior - (double)h_logq[j] - top);
            } else {
                for (uint64_t j = 0; j < m; ++j) h_wd[j] = 1.0;
            }
            double sw = 0.0, sw2 = 0.0;
            for (uint64_t j = 0; j < m; ++j) {
                sw += h_wd[j];
                sw2 += h_wd[j] * h_wd[j];
            }
            R.ess_fraction = sw2 > 0.0 ? sw * sw / sw2 / (double)m : 0.0;
            for (uint64_t j = 0; j < m; ++j) {
                h_wd[j] /= sw;
                h_w[j] = (float)h_wd[j];
            }
        }
        // the next round's proposal: train on this round's weighted accepts
        const bool last = r + 1 == cfg->rounds;
        if (last) {
            last_n = m;
            if (m > 0) {
                if (theta_out)
                    SMC_TRY(cudaMemcpyAsync(theta_out, acc_theta, sizeof(float) * 8 * m, cudaMemcpyDefault, s),
                            "cudaMemcpyAsync(theta)");
                if (dist_out)
                    SMC_TRY(cudaMemcpyAsync(dist_out, acc_dist, sizeof(double) * m, cudaMemcpyDefault, s),
                            "cudaMemcpyAsync(dist)");
                if (weight_out)
                    SMC_TRY(cudaMemcpyAsync(weight_out, h_wd.data(), sizeof(double) * m, cudaMemcpyDefault, s),
                            "cudaMemcpyAsync(weights)");
            }
            SMC_TRY(cudaEventRecord(gd.ev[3], s), "cudaEventRecord");
        } else {
            const bool trainable = m >= 64 && R.ess_fraction >= cfg->ess_min;
            if (trainable) {
                SMC_TRY(cudaMemcpyAsync(d_train, acc_theta, sizeof(float) * 8 * m, cudaMemcpyDeviceToDevice, s),
                        "cudaMemcpyAsync(training set)");
                SMC_TRY(cudaMemcpyAsync(d_w, h_w.data(), sizeof(float) * m, cudaMemcpyHostToDevice, s),
                        "cudaMemcpyAsync(weights)");
                float loss = 0.f;
                SMC_ST(abc_maf_train(gd.flow, m, d_train, d_w, cfg->train_steps, cfg->train_batch, cfg->train_lr,
                                     cfg->seed + 7919 * (uint64_t)r, &loss, s));
                R.train_loss = loss;
            }
            SMC_TRY(cudaEventRecord(gd.ev[3], s), "cudaEventRecord");
            use_flow = trainable;
        }
        SMC_TRY(cudaEventSynchronize(gd.ev[3]), "cudaEventSynchronize");
        cudaEventElapsedTime(&R.ms_propose, gd.ev[0], gd.ev[1]);
        cudaEventElapsedTime(&R.ms_simulate, gd.ev[1], gd.ev[2]);
        cudaEventElapsedTime(&R.ms_train, gd.ev[2], gd.ev[3]);
        eps *= cfg->eps_factor;
    }
    SMC_TRY(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    *n_out = last_n;
    return abcgb::plan_ok();
}
