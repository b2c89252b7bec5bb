// abc_pmc.cu -- plain sequential ABC: population Monte Carlo ABC (Beaumont,
// Cornuet, Marin, Robert 2009). Proposal and weight kernels plus the host loop
// over rounds; simulation and acceptance run in the batched rejection kernel
// of a one-region plan that reads the proposals (NaN rows skipped).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
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
abc_status plan_scratch_alloc(void** ptr, size_t bytes, cudaStream_t s);
}  // namespace abcgb

namespace {

using abcgb::plan_cuda_fail;
using abcgb::plan_fail;

struct Mat8 {
    float a[64];   // row-major
};

struct BoxF {
    float lo[8], hi[8];
};

// proposal j of index first + j: Philox blocks g = 0, 1 give 8 normals (four
// Box-Muller pairs), block g = 2 the parent uniform (stream 2)
__global__ void propose_kernel(const __grid_constant__ abcgb::ModelParams p, uint32_t ctr3, const float* __restrict__ old,
                               const double* __restrict__ cumw, uint64_t m, const __grid_constant__ Mat8 L,
                               const __grid_constant__ BoxF box, uint64_t first, uint64_t n, float* __restrict__ out)
{
    const uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const uint64_t i = first + j;
    const uint4 a = abcgb::rng_block_s(p, i, 0, ctr3, 0);
    const uint4 b = abcgb::rng_block_s(p, i, 0, ctr3, 1);
    const uint4 c = abcgb::rng_block_s(p, i, 0, ctr3, 2);
    float z[8];
    abcgb::box_muller<abcgb::kFast>(a.x, a.y, z[0], z[1]);
    abcgb::box_muller<abcgb::kFast>(a.z, a.w, z[2], z[3]);
    abcgb::box_muller<abcgb::kFast>(b.x, b.y, z[4], z[5]);
    abcgb::box_muller<abcgb::kFast>(b.z, b.w, z[6], z[7]);
    // 53-bit uniform from two words, then the inverse CDF of the weights
    const double u = ((double)(c.x >> 5) * 67108864.0 + (double)(c.y >> 6)) * 0x1p-53 * cumw[m - 1];
    uint64_t lo = 0, hi = m - 1;
    while (lo < hi) {
        const uint64_t mid = (lo + hi) / 2;
        if (cumw[mid] > u)
            hi = mid;
        else
            lo = mid + 1;
    }
    const float* par = old + 8 * lo;
    bool inside = true;
    float th[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        float v = par[r];
#pragma unroll
        for (int k = 0; k <= r; ++k) v = __fmaf_rn(L.a[r * 8 + k], z[k], v);
        th[r] = v;
        inside = inside && v >= box.lo[r] && v <= box.hi[r];
    }
    if (!inside) th[0] = __int_as_float(0x7FC00000);
    float4* o = reinterpret_cast<float4*>(out + 8 * j);
    o[0] = make_float4(th[0], th[1], th[2], th[3]);
    o[1] = make_float4(th[4], th[5], th[6], th[7]);
}

// a = L^-1 theta for each row (forward substitution)
__device__ __forceinline__ void whiten(const Mat8& Li, const float* th, float a[8])
{
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        float v = 0.f;
#pragma unroll
        for (int k = 0; k <= r; ++k) v = __fmaf_rn(Li.a[r * 8 + k], th[k], v);
        a[r] = v;
    }
}

constexpr int kTile = 256;

__global__ void __launch_bounds__(kTile) weights_kernel(const float* __restrict__ nw, uint64_t n,
                                                        const float* __restrict__ old, const double* __restrict__ w_old,
                                                        uint64_t m, const __grid_constant__ Mat8 Li,
                                                        double* __restrict__ out)
{
    __shared__ float bs[kTile][9];
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float a[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (i < n) whiten(Li, nw + 8 * i, a);
    double acc = 0.0;
    for (uint64_t base = 0; base < m; base += kTile) {
        const uint64_t jj = base + threadIdx.x;
        if (jj < m) {
            float b[8];
            whiten(Li, old + 8 * jj, b);
#pragma unroll
            for (int r = 0; r < 8; ++r) bs[threadIdx.x][r] = b[r];
            bs[threadIdx.x][8] = (float)w_old[jj];
        }
        __syncthreads();
        const int cnt = (int)(m - base < (uint64_t)kTile ? m - base : (uint64_t)kTile);
        float tile = 0.f;
        for (int q = 0; q < cnt; ++q) {
            float d2 = 0.f;
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const float d = a[r] - bs[q][r];
                d2 = __fmaf_rn(d, d, d2);
            }
            tile = __fmaf_rn(bs[q][8], __expf(-0.5f * d2), tile);
        }
        acc += (double)tile;
        __syncthreads();
    }
    if (i < n) out[i] = 1.0 / acc;
}

bool cholesky8(const double S[64], double L[64])
{
    std::memset(L, 0, 64 * sizeof(double));
    for (int r = 0; r < 8; ++r) {
        for (int c = 0; c <= r; ++c) {
            double v = S[r * 8 + c];
            for (int k = 0; k < c; ++k) v -= L[r * 8 + k] * L[c * 8 + k];
            if (r == c) {
                if (!(v > 0.0)) return false;
                L[r * 8 + r] = std::sqrt(v);
            } else {
                L[r * 8 + c] = v / L[c * 8 + c];
            }
        }
    }
    return true;
}

void invert_lower8(const double L[64], double Li[64])
{
    std::memset(Li, 0, 64 * sizeof(double));
    for (int c = 0; c < 8; ++c) {
        Li[c * 8 + c] = 1.0 / L[c * 8 + c];
        for (int r = c + 1; r < 8; ++r) {
            double v = 0.0;
            for (int k = c; k < r; ++k) v -= L[r * 8 + k] * Li[k * 8 + c];
            Li[r * 8 + c] = v / L[r * 8 + r];
        }
    }
}

Mat8 to_mat(const double* M)
{
    Mat8 m;
    for (int k = 0; k < 64; ++k) m.a[k] = (float)M[k];
    return m;
}

abc_status check_L(const float* L, double Ld[64])
{
    if (!L) return plan_fail(ABC_ERR_INVALID_ARG, "L is NULL");
    for (int r = 0; r < 8; ++r)
        for (int c = 0; c < 8; ++c) {
            Ld[r * 8 + c] = c <= r ? (double)L[r * 8 + c] : 0.0;
            if (r == c && !(L[r * 8 + c] > 0.f)) return plan_fail(ABC_ERR_INVALID_ARG, "L needs a positive diagonal");
        }
    return ABC_OK;
}

}  // namespace

#define PMC_TRY(expr, what)                                   \
    do {                                                      \
        cudaError_t _e = (expr);                              \
        if (_e != cudaSuccess) return plan_cuda_fail(_e, what); \
    } while (0)
#define PMC_ST(expr)                 \
    do {                             \
        abc_status _s = (expr);      \
        if (_s != ABC_OK) return _s; \
    } while (0)

namespace {

// cumulative weights (double) on the device for the inverse-CDF parent draw
abc_status upload_cumw(const std::vector<double>& w, double* d_cumw, cudaStream_t s, std::vector<double>& scratch)
{
    scratch.resize(w.size());
    double c = 0.0;
    for (size_t j = 0; j < w.size(); ++j) {
        c += w[j];
        scratch[j] = c;
    }
    PMC_TRY(cudaMemcpyAsync(d_cumw, scratch.data(), sizeof(double) * w.size(), cudaMemcpyHostToDevice, s),
            "cudaMemcpyAsync(cumw)");
    return ABC_OK;
}

}  // namespace

extern "C" {

abc_status abc_pmc_propose(const abc_prior_box* prior, const float* theta_old, const double* w_old, uint64_t m,
                           const float* L, uint64_t seed, uint64_t first_index, uint64_t n, float* theta_out,
                           void* cuda_stream)
{
    abc_status st;
    if (!abcgb::plan_check_prior(prior, &st)) return st;
    if (!theta_old || !w_old || m == 0 || (n && !theta_out)) return plan_fail(ABC_ERR_INVALID_ARG, "bad buffers");
    double Ld[64];
    if ((st = check_L(L, Ld)) != ABC_OK) return st;
    if (n == 0) return abcgb::plan_ok();
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // cumulative weights of the caller's device weights
    double* d_cumw = nullptr;
    if ((st = abcgb::plan_scratch_alloc(reinterpret_cast<void**>(&d_cumw), sizeof(double) * m, s)) != ABC_OK)
        return st;
    struct FreeOnReturn {   // every return below gives the scratch back, stream-ordered
        void* p;
        cudaStream_t s;
        ~FreeOnReturn() { cudaFreeAsync(p, s); }
    } release{d_cumw, s};
    std::vector<double> w(m), tmp;
    PMC_TRY(cudaMemcpyAsync(w.data(), w_old, sizeof(double) * m, cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync(w)");
    PMC_TRY(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    if ((st = upload_cumw(w, d_cumw, s, tmp)) != ABC_OK) return st;
    const abcgb::ModelParams p = abcgb::plan_make_params(prior, 1, 1, seed, 2, nullptr);
    BoxF box;
    for (int j = 0; j < 8; ++j) {
        box.lo[j] = prior->lo[j];
        box.hi[j] = prior->hi[j];
    }
    propose_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, 2u << 2, theta_old, d_cumw, m, to_mat(Ld), box,
                                                               first_index, n, theta_out);
    cudaError_t e = cudaGetLastError();
    PMC_TRY(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    PMC_TRY(e, "propose launch");
    return abcgb::plan_ok();
}

abc_status abc_pmc_weights(const float* theta_new, uint64_t n, const float* theta_old, const double* w_old,
                           uint64_t m, const float* L, double* w_out, void* cuda_stream)
{
    abc_status st;
    if (!theta_old || !w_old || m == 0 || (n && (!theta_new || !w_out)))
        return plan_fail(ABC_ERR_INVALID_ARG, "bad buffers");
    double Ld[64], Li[64];
    if ((st = check_L(L, Ld)) != ABC_OK) return st;
    if (n == 0) return abcgb::plan_ok();
    invert_lower8(Ld, Li);
    weights_kernel<<<(unsigned)((n + kTile - 1) / kTile), kTile, 0, (cudaStream_t)cuda_stream>>>(
        theta_new, n, theta_old, w_old, m, to_mat(Li), w_out);
    PMC_TRY(cudaGetLastError(), "weights launch");
    return abcgb::plan_ok();
}

abc_status abc_pmc_run(const abc_prior_box* prior, const int32_t* observed, int32_t T, int64_t N_pop,
                       const abc_pmc_config* cfg, abc_pmc_round* rounds_out, float* theta_out, double* weight_out,
                       double* dist_out, uint64_t* n_out, void* cuda_stream)
{
    abc_status st;
    if (!abcgb::plan_check_prior(prior, &st)) return st;
    if (!cfg || !rounds_out || !n_out) return plan_fail(ABC_ERR_INVALID_ARG, "cfg, rounds_out and n_out are required");
    if (cfg->rounds < 1 || cfg->n_particles < 2 || cfg->batch == 0 || cfg->max_batches < 1 ||
        cfg->capacity < cfg->n_particles || !(cfg->eps0 >= 0.0) || !(cfg->eps_factor > 0.0) || cfg->eps_factor > 1.0)
        return plan_fail(ABC_ERR_INVALID_ARG, "bad population Monte Carlo configuration");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (!s) return plan_fail(ABC_ERR_INVALID_ARG, "population Monte Carlo needs a non-default stream");
    const uint64_t B = cfg->batch, cap = cfg->capacity;
    std::vector<void*> owned;
    struct Free {
        std::vector<void*>& v;
        abc_plan plan = nullptr;
        ~Free()
        {
            for (void* q : v) cudaFree(q);
            if (plan) abc_plan_destroy(plan);
        }
    } guard{owned};
    float *d_prop = nullptr, *d_pop = nullptr, *d_new = nullptr;
    double *d_w = nullptr, *d_cumw = nullptr, *d_wnew = nullptr;
    PMC_TRY(cudaMalloc(&d_prop, sizeof(float) * 8 * B), "cudaMalloc");
    owned.push_back(d_prop);
    PMC_TRY(cudaMalloc(&d_pop, sizeof(float) * 8 * cap), "cudaMalloc");
    owned.push_back(d_pop);
    PMC_TRY(cudaMalloc(&d_new, sizeof(float) * 8 * cap), "cudaMalloc");
    owned.push_back(d_new);
    PMC_TRY(cudaMalloc(&d_w, sizeof(double) * cap), "cudaMalloc");
    owned.push_back(d_w);
    PMC_TRY(cudaMalloc(&d_cumw, sizeof(double) * cap), "cudaMalloc");
    owned.push_back(d_cumw);
    PMC_TRY(cudaMalloc(&d_wnew, sizeof(double) * cap), "cudaMalloc");
    owned.push_back(d_wnew);
    cudaEvent_t e0, e1;
    PMC_TRY(cudaEventCreate(&e0), "cudaEventCreate");
    PMC_TRY(cudaEventCreate(&e1), "cudaEventCreate");

    const abcgb::ModelParams pp = abcgb::plan_make_params(prior, 1, 1, cfg->seed, 2, nullptr);
    BoxF box;
    for (int j = 0; j < 8; ++j) {
        box.lo[j] = prior->lo[j];
        box.hi[j] = prior->hi[j];
    }
    std::vector<float> h_pop;
    std::vector<double> h_w, h_tmp;
    uint64_t m = 0;   // current population size
    double eps = cfg->eps0;
    double Ld[64], Li[64];
    for (int32_t r = 0; r < cfg->rounds; ++r) {
        abc_pmc_round& R = rounds_out[r];
        R = abc_pmc_round{};
        R.eps = eps;
        PMC_TRY(cudaEventRecord(e0, s), "cudaEventRecord");
        const uint64_t base = (uint64_t)r * (uint64_t)cfg->max_batches * B;
        if (r > 0) {
            // Sigma = 2 Cov_w of the population, L its Cholesky factor (jitter if needed)
            double mean[8] = {0}, S[64] = {0}, sw = 0.0;
            for (uint64_t j = 0; j < m; ++j) {
                sw += h_w[j];
                for (int a = 0; a < 8; ++a) mean[a] += h_w[j] * h_pop[8 * j + a];
            }
            for (int a = 0; a < 8; ++a) mean[a] /= sw;
            for (uint64_t j = 0; j < m; ++j)
                for (int a = 0; a < 8; ++a)
                    for (int b = 0; b <= a; ++b)
                        S[a * 8 + b] += h_w[j] * (h_pop[8 * j + a] - mean[a]) * (h_pop[8 * j + b] - mean[b]);
            double tr = 0.0;
            for (int a = 0; a < 8; ++a)
                for (int b = 0; b <= a; ++b) {
                    S[a * 8 + b] = 2.0 * S[a * 8 + b] / sw;
                    S[b * 8 + a] = S[a * 8 + b];
                }
            for (int a = 0; a < 8; ++a) tr += S[a * 9];
            bool okc = false;
            for (int k = 0; k < 12 && !okc; ++k) {
                double J[64];
                std::memcpy(J, S, sizeof J);
                for (int a = 0; a < 8; ++a) J[a * 9] += (k ? tr / 8.0 * 1e-12 * std::pow(10.0, k) : 0.0);
                okc = cholesky8(J, Ld);
            }
            if (!okc) return plan_fail(ABC_ERR_INVALID_ARG, "population covariance is not positive definite");
            invert_lower8(Ld, Li);
            PMC_TRY(cudaMemcpyAsync(d_pop, h_pop.data(), sizeof(float) * 8 * m, cudaMemcpyHostToDevice, s), "upload");
            PMC_TRY(cudaMemcpyAsync(d_w, h_w.data(), sizeof(double) * m, cudaMemcpyHostToDevice, s), "upload");
            PMC_ST(upload_cumw(h_w, d_cumw, s, h_tmp));
        }
        // one plan for every round, made in the first; a round sets its eps,
        // proposal buffer and first index and clears the accepted samples
        if (!guard.plan) {
            abc_region reg{};
            reg.observed = observed;
            reg.T = T;
            reg.N_pop = N_pop;
            reg.eps = eps;
            reg.n_samples = B;
            reg.first_index = base;
            reg.stream = 0;
            reg.capacity = cap;
            reg.theta_in = nullptr;
            PMC_ST(abc_plan_create(prior, &reg, 1, cfg->seed, cfg->mode, &guard.plan));
        }
        PMC_ST(abc_plan_set_eps(guard.plan, 0, eps));
        PMC_ST(abc_plan_set_region(guard.plan, 0, r > 0 ? d_prop : nullptr, base));
        PMC_ST(abc_plan_reset(guard.plan, s));
        uint64_t n_acc = 0, batches = 0;
        while (n_acc < cfg->n_particles && batches < (uint64_t)cfg->max_batches) {
            if (r > 0)
                propose_kernel<<<(unsigned)((B + 255) / 256), 256, 0, s>>>(pp, 2u << 2, d_pop, d_cumw, m, to_mat(Ld),
                                                                           box, base + batches * B, B, d_prop);
            PMC_TRY(cudaGetLastError(), "propose launch");
            PMC_ST(abc_plan_run(guard.plan, s));
            ++batches;
            PMC_ST(abc_plan_results(guard.plan, 0, &n_acc, nullptr, nullptr, nullptr, nullptr, s));
        }
        R.n_sims = batches * B;
        float* acc_theta = nullptr;
        double* acc_dist = nullptr;
        uint64_t* acc_idx = nullptr;
        PMC_ST(abc_plan_results(guard.plan, 0, &n_acc, nullptr, &acc_theta, &acc_dist, &acc_idx, s));
        const uint64_t mm = std::min(n_acc, cap);
        R.n_accepted = mm;
        if (mm < 2) return plan_fail(ABC_ERR_INVALID_ARG, "a round accepted fewer than 2 particles");
        std::vector<double> w_slot(mm, 1.0), dist_slot(mm);
        std::vector<float> pop_slot(8 * mm);
        std::vector<uint64_t> idx_slot(mm);
        if (r > 0) {
            PMC_TRY(cudaMemcpyAsync(d_new, acc_theta, sizeof(float) * 8 * mm, cudaMemcpyDeviceToDevice, s), "copy");
            weights_kernel<<<(unsigned)((mm + kTile - 1) / kTile), kTile, 0, s>>>(d_new, mm, d_pop, d_w, m, to_mat(Li),
                                                                              d_wnew);
            PMC_TRY(cudaGetLastError(), "weights launch");
            PMC_TRY(cudaMemcpyAsync(w_slot.data(), d_wnew, sizeof(double) * mm, cudaMemcpyDeviceToHost, s), "download");
        }
        PMC_TRY(cudaMemcpyAsync(pop_slot.data(), acc_theta, sizeof(float) * 8 * mm, cudaMemcpyDeviceToHost, s),
                "download");
        PMC_TRY(cudaMemcpyAsync(dist_slot.data(), acc_dist, sizeof(double) * mm, cudaMemcpyDeviceToHost, s), "download");
        PMC_TRY(cudaMemcpyAsync(idx_slot.data(), acc_idx, sizeof(uint64_t) * mm, cudaMemcpyDeviceToHost, s), "download");
        PMC_TRY(cudaStreamSynchronize(s), "cudaStreamSynchronize");
        // the population in ascending sample index: the plan's accept slots
        // follow the order of its atomics, which changes from run to run, and
        // the next round's resampling (by cumulative weight) and every sum
        // below follow the population's order; so a seed fixes the whole run
        std::vector<uint32_t> ord(mm);
        for (uint64_t j = 0; j < mm; ++j) ord[j] = (uint32_t)j;
        std::sort(ord.begin(), ord.end(), [&](uint32_t a, uint32_t b) { return idx_slot[a] < idx_slot[b]; });
        std::vector<float> pop(8 * mm);
        std::vector<double> w_new(mm), dist(mm);
        for (uint64_t j = 0; j < mm; ++j) {
            std::memcpy(&pop[8 * j], &pop_slot[8 * (size_t)ord[j]], 8 * sizeof(float));
            w_new[j] = w_slot[ord[j]];
            dist[j] = dist_slot[ord[j]];
        }
        double sw = 0.0, sw2 = 0.0;
        for (double v : w_new) {
            sw += v;
            sw2 += v * v;
        }
        for (double& v : w_new) v /= sw;
        R.ess_fraction = sw * sw / sw2 / (double)mm;
        h_pop.swap(pop);
        h_w.swap(w_new);
        m = mm;
        if (r + 1 == cfg->rounds) {
            if (theta_out)
                PMC_TRY(cudaMemcpyAsync(theta_out, h_pop.data(), sizeof(float) * 8 * m, cudaMemcpyDefault, s), "out");
            if (dist_out)
                PMC_TRY(cudaMemcpyAsync(dist_out, dist.data(), sizeof(double) * m, cudaMemcpyDefault, s), "out");
            if (weight_out)
                PMC_TRY(cudaMemcpyAsync(weight_out, h_w.data(), sizeof(double) * m, cudaMemcpyDefault, s), "out");
        }
        PMC_TRY(cudaEventRecord(e1, s), "cudaEventRecord");
        PMC_TRY(cudaEventSynchronize(e1), "cudaEventSynchronize");
        cudaEventElapsedTime(&R.ms, e0, e1);
        eps *= cfg->eps_factor;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    PMC_TRY(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    *n_out = m;
    return abcgb::plan_ok();
}

}  // extern "C"
