// abc_api.cu -- the C ABI declared in include/abc_gb300.h: argument checks,
// kernel parameters, stream-ordered scratch memory and error reporting.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/abc_gb300.h"
#include "abc_kernels.h"
#include "abc_model.cuh"

namespace {

thread_local std::string g_last_error;
thread_local uint64_t g_last_sim_days = 0;

abc_status fail(abc_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

abc_status ok()
{
    g_last_error.clear();
    return ABC_OK;
}

abc_status cuda_fail(cudaError_t e, const char* what)
{
    return fail(e == cudaErrorMemoryAllocation ? ABC_ERR_NOMEM : ABC_ERR_CUDA, "%s: %s (%s)", what,
                cudaGetErrorString(e), cudaGetErrorName(e));
}

// Host-side fault injection for tests of the error paths: the environment
// variable ABC_GB300_INJECT_FAULT=alloc|launch makes the next scratch
// allocation or kernel launch report failure without touching the GPU.
bool injected(const char* what)
{
    const char* v = std::getenv("ABC_GB300_INJECT_FAULT");
    return v && std::strcmp(v, what) == 0;
}

#define CUDA_TRY(expr, what)                        \
    do {                                            \
        cudaError_t _e = (expr);                    \
        if (_e != cudaSuccess) return cuda_fail(_e, what); \
    } while (0)

abc_status check_prior(const abc_prior_box* prior)
{
    if (!prior) return fail(ABC_ERR_INVALID_ARG, "prior is NULL");
    for (int j = 0; j < 8; ++j) {
        if (!std::isfinite(prior->lo[j]) || !std::isfinite(prior->hi[j]))
            return fail(ABC_ERR_INVALID_ARG, "prior bound %d is not finite", j);
        if (prior->lo[j] > prior->hi[j]) return fail(ABC_ERR_INVALID_ARG, "prior lo[%d] > hi[%d]", j, j);
        if (!std::isfinite(prior->hi[j] - prior->lo[j]))
            return fail(ABC_ERR_INVALID_ARG, "prior width %d overflows float", j);
    }
    return ABC_OK;
}

abc_status check_model(int32_t T, int64_t N_pop, uint32_t stream)
{
    if (T < 1 || T > ABC_T_MAX) return fail(ABC_ERR_INVALID_ARG, "T = %d outside [1, %d]", T, ABC_T_MAX);
    if (N_pop < 1 || N_pop >= ((int64_t)1 << 31))
        return fail(ABC_ERR_INVALID_ARG, "N_pop = %lld outside [1, 2^31)", (long long)N_pop);
    if (stream > ABC_STREAM_MAX) return fail(ABC_ERR_INVALID_ARG, "stream = %u above 2^30 - 1", stream);
    return ABC_OK;
}

abc_status check_initial(const int32_t* ard, int64_t N_pop)
{
    if (!ard) return fail(ABC_ERR_INVALID_ARG, "initial condition is NULL");
    if (ard[0] < 0 || ard[1] < 0 || ard[2] < 0) return fail(ABC_ERR_INVALID_ARG, "negative initial count");
    if ((int64_t)ard[0] + ard[1] + ard[2] > N_pop)
        return fail(ABC_ERR_INVALID_ARG, "A0 + R0 + D0 exceeds N_pop");
    return ABC_OK;
}

// Kernel parameters: prior, Philox round keys, population constants.
abcgb::ModelParams make_params(const abc_prior_box* prior, int32_t T, int64_t N_pop, uint64_t seed, uint32_t stream,
                               const int32_t* ard0)
{
    abcgb::ModelParams p;
    std::memset(&p, 0, sizeof p);
    if (prior) {
        for (int j = 0; j < 8; ++j) {
            p.lo[j] = prior->lo[j];
            volatile float w = prior->hi[j] - prior->lo[j];   // one IEEE binary32 subtraction
            p.width[j] = w;
        }
    }
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        p.rk0[r] = k0;
        p.rk1[r] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    p.ctr3_base = stream << 2;
    p.T = T;
    p.P = (int32_t)N_pop;
    volatile float pf = (float)N_pop;
    volatile float inv = 1.0f / pf;
    p.inv_p = inv;
    if (ard0) {
        p.A0 = ard0[0];
        p.R0 = ard0[1];
        p.D0 = ard0[2];
        p.room0 = (int32_t)(N_pop - ((int64_t)ard0[0] + ard0[1] + ard0[2]));
    }
    return p;
}

// The public mode (ABC_EXACT or ABC_FAST, optionally | ABC_VARIANCE_LITERAL)
// and the kernels' mode bits.
bool valid_mode(abc_mode mode)
{
    const int base = (int)mode & ~(int)ABC_VARIANCE_LITERAL;
    return base == ABC_EXACT || base == ABC_FAST;
}

int kernel_mode(abc_mode mode)
{
    return (((int)mode & ABC_FAST) ? abcgb::kFast : abcgb::kExact) |
           (((int)mode & ABC_VARIANCE_LITERAL) ? abcgb::kLiteral : 0);
}

// Observed [3][T+1] rows A, R, D -> per-day int4 (A, R, D, 0).
abc_status pack_observed(const int32_t* observed, int32_t T, int64_t N_pop, std::vector<int4>& out)
{
    if (!observed) return fail(ABC_ERR_INVALID_ARG, "observed is NULL");
    out.resize((size_t)T + 1);
    for (int32_t d = 0; d <= T; ++d) {
        const int32_t A = observed[d], R = observed[(T + 1) + d], D = observed[2 * (T + 1) + d];
        if (A < 0 || R < 0 || D < 0) return fail(ABC_ERR_INVALID_ARG, "negative observed count on day %d", d);
        out[d] = make_int4(A, R, D, 0);
    }
    const int32_t ard0[3] = {out[0].x, out[0].y, out[0].z};
    return check_initial(ard0, N_pop);
}

// Largest integer distance^2 whose distance sqrt((double)a) is <= eps. The
// predicate is monotone in a, so a binary search over [0, 2^63] is exact.
uint64_t acc_threshold(double eps)
{
    const uint64_t cap = 0x8000000000000000ull;
    if (std::sqrt((double)cap) <= eps) return cap;
    uint64_t lo = 0, hi = cap;   // sqrt(lo) <= eps (eps >= 0), sqrt(hi) > eps
    while (hi - lo > 1) {
        const uint64_t mid = lo + (hi - lo) / 2;
        if (std::sqrt((double)mid) <= eps)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

struct Scratch {
    void* ptr = nullptr;
    cudaStream_t s = nullptr;
    ~Scratch()
    {
        if (ptr) cudaFreeAsync(ptr, s);
    }
};

constexpr int kMaxCachedDevices = 64;

// Stream-ordered scratch comes from one memory pool per device that keeps up
// to kPoolKeepBytes of freed memory mapped across synchronisations. (The
// device's default pool gives all freed memory back at every synchronisation,
// so each call mapped its scratch anew: about 150 us of host time per call,
// and as much again at the caller's next synchronisation.) A pool is created
// on a device's first use and kept for the life of the process; a failed
// creation is not cached, so a later call tries again.
constexpr uint64_t kPoolKeepBytes = 1ull << 30;
std::mutex g_pool_mutex;
cudaMemPool_t g_pools[kMaxCachedDevices] = {};

abc_status scratch_pool(cudaMemPool_t* out)
{
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev < 0 || dev >= kMaxCachedDevices) return fail(ABC_ERR_INVALID_ARG, "device ordinal %d too large", dev);
    std::lock_guard<std::mutex> lock(g_pool_mutex);
    if (!g_pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        CUDA_TRY(cudaMemPoolCreate(&pool, &props), "cudaMemPoolCreate");
        uint64_t keep = kPoolKeepBytes;
        const cudaError_t e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) {
            cudaMemPoolDestroy(pool);
            return cuda_fail(e, "cudaMemPoolSetAttribute(release threshold)");
        }
        g_pools[dev] = pool;
    }
    *out = g_pools[dev];
    return ABC_OK;
}

abc_status alloc_scratch(Scratch& sc, size_t bytes, cudaStream_t s)
{
    sc.s = s;
    if (injected("alloc")) return fail(ABC_ERR_NOMEM, "scratch allocation failed (injected)");
    cudaMemPool_t pool = nullptr;
    abc_status st = scratch_pool(&pool);
    if (st != ABC_OK) return st;
    cudaError_t e = cudaMallocFromPoolAsync(&sc.ptr, bytes, pool, s);
    if (e != cudaSuccess) {
        sc.ptr = nullptr;
        return cuda_fail(e, "cudaMallocFromPoolAsync(scratch)");
    }
    return ABC_OK;
}

// Per-thread, per-device scratch of abc_sample: device memory for the observed
// series and counters, pinned host memory to stage them. Kept across calls and
// grown when a longer series needs more; abc_sample synchronizes its stream
// before returning, so the next call on this thread can reuse it.
struct SampleScratch {
    void* dev = nullptr;
    void* host = nullptr;
    size_t bytes = 0;
};

thread_local SampleScratch g_sample_scratch[kMaxCachedDevices];

abc_status sample_scratch(size_t bytes, SampleScratch** out)
{
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev < 0 || dev >= kMaxCachedDevices) return fail(ABC_ERR_INVALID_ARG, "device ordinal %d too large", dev);
    SampleScratch& sc = g_sample_scratch[dev];
    if (sc.bytes < bytes) {
        if (injected("alloc")) return fail(ABC_ERR_NOMEM, "scratch allocation failed (injected)");
        if (sc.dev) cudaFree(sc.dev);
        if (sc.host) cudaFreeHost(sc.host);
        sc = SampleScratch();
        void* d = nullptr;
        void* h = nullptr;
        CUDA_TRY(cudaMalloc(&d, bytes), "cudaMalloc(scratch)");
        cudaError_t e = cudaMallocHost(&h, bytes);
        if (e != cudaSuccess) {
            cudaFree(d);
            return cuda_fail(e, "cudaMallocHost(staging)");
        }
        sc.dev = d;
        sc.host = h;
        sc.bytes = bytes;
    } else if (injected("alloc")) {
        return fail(ABC_ERR_NOMEM, "scratch allocation failed (injected)");
    }
    *out = &sc;
    return ABC_OK;
}

}  // namespace

// A region's observed series on the device (abc_observed_create).
struct abc_observed_s {
    int device = 0;
    int32_t T = 0;
    int64_t N_pop = 0;
    int32_t ard0[3] = {0, 0, 0};
    void* dev = nullptr;   // int4 [T+1] (A, R, D, 0)
};

// Scratch of abc_sample_noalloc: bytes [0, 24) hold the three counters
// (accepts, claimed indices, simulated days), bytes [256, 256 + 16 (T+1)) the
// observed series. Host code must not pass this name to a kernel (on the host
// it is a stand-in, not a device address); noalloc_scratch() returns the
// device address.
static __device__ __align__(256) unsigned char abc_noalloc_scratch[ABC_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kNoallocMaxDevices = 256;

struct NoallocDevice {
    std::mutex mu;
    void* ptr = nullptr;   // set once a lookup on this device has succeeded
};

NoallocDevice g_noalloc_devices[kNoallocMaxDevices];

// Device address of abc_noalloc_scratch on the current device, looked up with
// that device current. A successful lookup is kept for the life of the
// process; a failed one is not, so a later call retries it.
abc_status noalloc_scratch(void** out)
{
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev < 0 || dev >= kNoallocMaxDevices) return fail(ABC_ERR_INVALID_ARG, "device ordinal %d too large", dev);
    NoallocDevice& d = g_noalloc_devices[dev];
    std::lock_guard<std::mutex> lock(d.mu);
    if (!d.ptr) {
        void* p = nullptr;
        CUDA_TRY(cudaGetSymbolAddress(&p, abc_noalloc_scratch), "cudaGetSymbolAddress(abc_noalloc_scratch)");
        d.ptr = p;
    }
    *out = d.ptr;
    return ABC_OK;
}

}  // namespace

namespace abcgb {
// Helpers shared with the batched-regions ABI (abc_plan.cu): the same error
// reporting, checks and kernel parameters as the calls in this file.
abc_status plan_fail(abc_status st, const char* msg) { return fail(st, "%s", msg); }
abc_status plan_cuda_fail(cudaError_t e, const char* what) { return cuda_fail(e, what); }
abc_status plan_ok() { return ok(); }
bool plan_check_prior(const abc_prior_box* prior, abc_status* st)
{
    *st = check_prior(prior);
    return *st == ABC_OK;
}
uint64_t plan_acc_threshold(double eps) { return acc_threshold(eps); }
// stream-ordered scratch from the per-device pool of this file (alloc_scratch);
// free it with cudaFreeAsync
abc_status plan_scratch_alloc(void** ptr, size_t bytes, cudaStream_t s)
{
    *ptr = nullptr;
    cudaMemPool_t pool = nullptr;
    const abc_status st = scratch_pool(&pool);
    if (st != ABC_OK) return st;
    const cudaError_t e = cudaMallocFromPoolAsync(ptr, bytes, pool, s);
    if (e != cudaSuccess) {
        *ptr = nullptr;
        return cuda_fail(e, "cudaMallocFromPoolAsync(scratch)");
    }
    return ABC_OK;
}
ModelParams plan_make_params(const abc_prior_box* prior, int32_t T, int64_t N_pop, uint64_t seed, uint32_t stream,
                             const int32_t* ard0)
{
    return make_params(prior, T, N_pop, seed, stream, ard0);
}
}  // namespace abcgb

extern "C" {

abc_status abc_sample(const abc_prior_box* prior, const int32_t* observed, int32_t T, int64_t N_pop, double eps,
                      uint64_t n_samples, uint64_t seed, uint32_t stream, abc_mode mode, uint64_t first_index,
                      float* theta_out, double* dist_out, uint64_t* idx_out, uint64_t capacity,
                      uint64_t* n_accepted, void* cuda_stream)
{
    abc_status st;
    if ((st = check_prior(prior)) != ABC_OK) return st;
    if ((st = check_model(T, N_pop, stream)) != ABC_OK) return st;
    if (!valid_mode(mode)) return fail(ABC_ERR_INVALID_ARG, "unknown mode %d", (int)mode);
    if (!(eps >= 0.0)) return fail(ABC_ERR_INVALID_ARG, "eps must be >= 0 and not NaN");
    if (!n_accepted) return fail(ABC_ERR_INVALID_ARG, "n_accepted is NULL");
    if (capacity > 0 && (!theta_out || !dist_out || !idx_out))
        return fail(ABC_ERR_INVALID_ARG, "output buffers are NULL");
    if (n_samples > ~(uint64_t)0 - first_index)
        return fail(ABC_ERR_INVALID_ARG, "first_index + n_samples overflows");
    std::vector<int4> obs;
    if ((st = pack_observed(observed, T, N_pop, obs)) != ABC_OK) return st;
    *n_accepted = 0;
    g_last_sim_days = 0;
    if (n_samples == 0) return ok();

    const int32_t ard0[3] = {obs[0].x, obs[0].y, obs[0].z};
    const abcgb::ModelParams p = make_params(prior, T, N_pop, seed, stream, ard0);
    cudaStream_t s = (cudaStream_t)cuda_stream;

    // scratch: three counters (accepts, claimed indices, simulated days), then
    // the observed series; staged through pinned host memory
    const size_t obs_off = 256;
    SampleScratch* sc = nullptr;
    if ((st = sample_scratch(obs_off + sizeof(int4) * obs.size(), &sc)) != ABC_OK) return st;
    unsigned long long* count_h = (unsigned long long*)sc->host;
    count_h[0] = count_h[1] = count_h[2] = 0;
    std::memcpy((char*)sc->host + obs_off, obs.data(), sizeof(int4) * obs.size());
    unsigned long long* count_d = (unsigned long long*)sc->dev;
    int4* obs_d = (int4*)((char*)sc->dev + obs_off);
    if (injected("launch")) return fail(ABC_ERR_CUDA, "kernel launch failed (injected)");
    // from here on the pinned staging buffer may be in use by the stream: every
    // error return first waits for the stream so the next call can reuse it
    auto drain = [s](abc_status e) {
        cudaStreamSynchronize(s);
        return e;
    };
    cudaError_t ce = cudaMemcpyAsync(sc->dev, sc->host, obs_off + sizeof(int4) * obs.size(), cudaMemcpyHostToDevice, s);
    if (ce != cudaSuccess) return drain(cuda_fail(ce, "cudaMemcpyAsync(observed, counters)"));

    abcgb::RejectArgs a;
    a.obs = obs_d;
    a.first_index = first_index;
    a.n_samples = n_samples;
    a.acc_max = acc_threshold(eps);
    a.count = count_d;
    a.next = count_d + 1;
    a.sim_days = count_d + 2;
    a.capacity = capacity;
    a.theta_out = theta_out;
    a.dist_out = dist_out;
    a.idx_out = idx_out;
    ce = abcgb::launch_reject(p, a, kernel_mode(mode), s, nullptr);
    if (ce != cudaSuccess) return drain(cuda_fail(ce, "abc_reject_kernel launch"));
    ce = cudaMemcpyAsync(count_h, count_d, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
    if (ce != cudaSuccess) return drain(cuda_fail(ce, "cudaMemcpyAsync(counters)"));
    CUDA_TRY(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    const unsigned long long count = count_h[0];
    g_last_sim_days = count_h[2];
    *n_accepted = count;
    if (count > capacity)
        return fail(ABC_ERR_CAPACITY, "%llu samples accepted, capacity %llu", count, (unsigned long long)capacity);
    return ok();
}

abc_status abc_observed_create(const int32_t* observed, int32_t T, int64_t N_pop, abc_observed* out)
{
    abc_status st;
    if (!out) return fail(ABC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if ((st = check_model(T, N_pop, 0)) != ABC_OK) return st;
    std::vector<int4> obs;
    if ((st = pack_observed(observed, T, N_pop, obs)) != ABC_OK) return st;
    abc_observed_s* o = new abc_observed_s();
    o->T = T;
    o->N_pop = N_pop;
    o->ard0[0] = obs[0].x;
    o->ard0[1] = obs[0].y;
    o->ard0[2] = obs[0].z;
    cudaError_t e = cudaGetDevice(&o->device);
    if (e == cudaSuccess) e = cudaMalloc(&o->dev, sizeof(int4) * obs.size());
    if (e == cudaSuccess) e = cudaMemcpy(o->dev, obs.data(), sizeof(int4) * obs.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        if (o->dev) cudaFree(o->dev);
        delete o;
        return cuda_fail(e, "observed series upload");
    }
    *out = o;
    return ok();
}

abc_status abc_observed_destroy(abc_observed obs)
{
    if (!obs) return fail(ABC_ERR_INVALID_ARG, "observed handle is NULL");
    cudaError_t e = cudaDeviceSynchronize();
    cudaFree(obs->dev);
    delete obs;
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
    return ok();
}

abc_status abc_sample_async(const abc_prior_box* prior, abc_observed obs, double eps, uint64_t n_samples,
                            uint64_t seed, uint32_t stream, abc_mode mode, uint64_t first_index, float* theta_out,
                            double* dist_out, uint64_t* idx_out, uint64_t capacity, uint64_t* counters_dev,
                            void* cuda_stream)
{
    abc_status st;
    if ((st = check_prior(prior)) != ABC_OK) return st;
    if (!obs) return fail(ABC_ERR_INVALID_ARG, "observed handle is NULL");
    if ((st = check_model(obs->T, obs->N_pop, stream)) != ABC_OK) return st;
    if (!valid_mode(mode)) return fail(ABC_ERR_INVALID_ARG, "unknown mode %d", (int)mode);
    if (!(eps >= 0.0)) return fail(ABC_ERR_INVALID_ARG, "eps must be >= 0 and not NaN");
    if (!counters_dev) return fail(ABC_ERR_INVALID_ARG, "counters_dev is NULL");
    if (capacity > 0 && (!theta_out || !dist_out || !idx_out))
        return fail(ABC_ERR_INVALID_ARG, "output buffers are NULL");
    if (n_samples > ~(uint64_t)0 - first_index)
        return fail(ABC_ERR_INVALID_ARG, "first_index + n_samples overflows");
    int dev = -1;
    CUDA_TRY(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev != obs->device) return fail(ABC_ERR_INVALID_ARG, "the observed handle belongs to another device");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    CUDA_TRY(cudaMemsetAsync(counters_dev, 0, 3 * sizeof(uint64_t), s), "cudaMemsetAsync(counters)");
    if (n_samples == 0) return ok();
    const abcgb::ModelParams p = make_params(prior, obs->T, obs->N_pop, seed, stream, obs->ard0);
    abcgb::RejectArgs a;
    a.obs = (const int4*)obs->dev;
    a.first_index = first_index;
    a.n_samples = n_samples;
    a.acc_max = acc_threshold(eps);
    unsigned long long* c = reinterpret_cast<unsigned long long*>(counters_dev);
    a.count = c;
    a.next = c + 1;
    a.sim_days = c + 2;
    a.capacity = capacity;
    a.theta_out = theta_out;
    a.dist_out = dist_out;
    a.idx_out = idx_out;
    if (injected("launch")) return fail(ABC_ERR_CUDA, "kernel launch failed (injected)");
    CUDA_TRY(abcgb::launch_reject(p, a, kernel_mode(mode), s, nullptr), "abc_reject_kernel launch");
    return ok();
}

abc_status abc_sample_until(const abc_prior_box* prior, abc_observed obs, double eps, uint64_t n_target,
                            uint64_t batch, uint64_t max_samples, uint64_t seed, uint32_t stream, abc_mode mode,
                            uint64_t first_index, float* theta_out, double* dist_out, uint64_t* idx_out,
                            uint64_t capacity, uint64_t* n_accepted, uint64_t* n_used, void* cuda_stream)
{
    abc_status st;
    if ((st = check_prior(prior)) != ABC_OK) return st;
    if (!obs) return fail(ABC_ERR_INVALID_ARG, "observed handle is NULL");
    if ((st = check_model(obs->T, obs->N_pop, stream)) != ABC_OK) return st;
    if (!valid_mode(mode)) return fail(ABC_ERR_INVALID_ARG, "unknown mode %d", (int)mode);
    if (!(eps >= 0.0)) return fail(ABC_ERR_INVALID_ARG, "eps must be >= 0 and not NaN");
    if (!n_accepted || !n_used) return fail(ABC_ERR_INVALID_ARG, "n_accepted and n_used are required");
    if (batch == 0) return fail(ABC_ERR_INVALID_ARG, "batch must be >= 1");
    if (capacity > 0 && (!theta_out || !dist_out || !idx_out))
        return fail(ABC_ERR_INVALID_ARG, "output buffers are NULL");
    if (max_samples > ~(uint64_t)0 - first_index)
        return fail(ABC_ERR_INVALID_ARG, "first_index + max_samples overflows");
    int dev = -1;
    CUDA_TRY(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev != obs->device) return fail(ABC_ERR_INVALID_ARG, "the observed handle belongs to another device");
    *n_accepted = 0;
    *n_used = 0;
    g_last_sim_days = 0;
    if (n_target == 0 || max_samples == 0) return ok();

    const abcgb::ModelParams p = make_params(prior, obs->T, obs->N_pop, seed, stream, obs->ard0);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    SampleScratch* sc = nullptr;
    if ((st = sample_scratch(256, &sc)) != ABC_OK) return st;
    unsigned long long* count_h = (unsigned long long*)sc->host;
    unsigned long long* count_d = (unsigned long long*)sc->dev;
    auto drain = [s](abc_status e) {
        cudaStreamSynchronize(s);
        return e;
    };
    // accepts and simulated days accumulate over the batches; each batch
    // starts its own index claims at 0
    cudaError_t ce = cudaMemsetAsync(count_d, 0, 3 * sizeof(unsigned long long), s);
    if (ce != cudaSuccess) return drain(cuda_fail(ce, "cudaMemsetAsync(counters)"));
    abcgb::RejectArgs a;
    a.obs = (const int4*)obs->dev;
    a.acc_max = acc_threshold(eps);
    a.count = count_d;
    a.next = count_d + 1;
    a.sim_days = count_d + 2;
    a.capacity = capacity;
    a.theta_out = theta_out;
    a.dist_out = dist_out;
    a.idx_out = idx_out;
    uint64_t used = 0;
    unsigned long long count = 0;
    while (used < max_samples && count < n_target && count <= capacity) {
        const uint64_t nb = std::min(batch, max_samples - used);
        if (used > 0) {
            ce = cudaMemsetAsync(count_d + 1, 0, sizeof(unsigned long long), s);
            if (ce != cudaSuccess) return drain(cuda_fail(ce, "cudaMemsetAsync(claim counter)"));
        }
        a.first_index = first_index + used;
        a.n_samples = nb;
        if (injected("launch")) return drain(fail(ABC_ERR_CUDA, "kernel launch failed (injected)"));
        ce = abcgb::launch_reject(p, a, kernel_mode(mode), s, nullptr);
        if (ce != cudaSuccess) return drain(cuda_fail(ce, "abc_reject_kernel launch"));
        ce = cudaMemcpyAsync(count_h, count_d, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
        if (ce != cudaSuccess) return drain(cuda_fail(ce, "cudaMemcpyAsync(counters)"));
        CUDA_TRY(cudaStreamSynchronize(s), "cudaStreamSynchronize");
        used += nb;
        count = count_h[0];
        g_last_sim_days = count_h[2];
    }
    *n_accepted = count;
    *n_used = used;
    if (count > capacity)
        return fail(ABC_ERR_CAPACITY, "%llu samples accepted, capacity %llu", count, (unsigned long long)capacity);
    return ok();
}

abc_status abc_distances(const abc_prior_box* prior, const int32_t* observed, int32_t T, int64_t N_pop,
                         uint64_t n_samples, uint64_t seed, uint32_t stream, abc_mode mode, uint64_t first_index,
                         double* dist_out, float* theta_out, void* cuda_stream)
{
    abc_status st;
    if ((st = check_prior(prior)) != ABC_OK) return st;
    if ((st = check_model(T, N_pop, stream)) != ABC_OK) return st;
    if (!valid_mode(mode)) return fail(ABC_ERR_INVALID_ARG, "unknown mode %d", (int)mode);
    if (n_samples > 0 && !dist_out) return fail(ABC_ERR_INVALID_ARG, "dist_out is NULL");
    if (n_samples > ~(uint64_t)0 - first_index)
        return fail(ABC_ERR_INVALID_ARG, "first_index + n_samples overflows");
    std::vector<int4> obs;
    if ((st = pack_observed(observed, T, N_pop, obs)) != ABC_OK) return st;
    if (n_samples == 0) return ok();
    const int32_t ard0[3] = {obs[0].x, obs[0].y, obs[0].z};
    const abcgb::ModelParams p = make_params(prior, T, N_pop, seed, stream, ard0);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    Scratch sc;
    if ((st = alloc_scratch(sc, sizeof(int4) * obs.size(), s)) != ABC_OK) return st;
    CUDA_TRY(cudaMemcpyAsync(sc.ptr, obs.data(), sizeof(int4) * obs.size(), cudaMemcpyHostToDevice, s),
             "cudaMemcpyAsync(observed)");
    abcgb::DistanceArgs a;
    a.obs = (const int4*)sc.ptr;
    a.first_index = first_index;
    a.n_samples = n_samples;
    a.dist_out = dist_out;
    a.theta_out = theta_out;
    if (injected("launch")) return fail(ABC_ERR_CUDA, "kernel launch failed (injected)");
    CUDA_TRY(abcgb::launch_distances(p, a, kernel_mode(mode), s), "abc_distance_kernel launch");
    return ok();
}

abc_status abc_simulate(const float* theta, const uint64_t* sample_index, uint64_t B, const int32_t* init_ard,
                        int32_t T, int64_t N_pop, uint64_t seed, uint32_t stream, abc_mode mode, int32_t* traj_out,
                        void* cuda_stream)
{
    abc_status st;
    if ((st = check_model(T, N_pop, stream)) != ABC_OK) return st;
    if (!valid_mode(mode)) return fail(ABC_ERR_INVALID_ARG, "unknown mode %d", (int)mode);
    if ((st = check_initial(init_ard, N_pop)) != ABC_OK) return st;
    if (B > 0 && (!theta || !sample_index || !traj_out)) return fail(ABC_ERR_INVALID_ARG, "NULL device buffer");
    if (B == 0) return ok();
    const abcgb::ModelParams p = make_params(nullptr, T, N_pop, seed, stream, init_ard);
    abcgb::SimulateArgs a;
    a.theta = theta;
    a.sample_index = sample_index;
    a.B = B;
    a.traj_out = traj_out;
    if (injected("launch")) return fail(ABC_ERR_CUDA, "kernel launch failed (injected)");
    CUDA_TRY(abcgb::launch_simulate(p, a, kernel_mode(mode), (cudaStream_t)cuda_stream), "abc_simulate_kernel launch");
    return ok();
}

abc_status abc_step(const float* theta, const int32_t* state_in, const uint64_t* sample_index, const int32_t* day,
                    uint64_t B, int64_t N_pop, uint64_t seed, uint32_t stream, abc_mode mode, int32_t* state_out,
                    int32_t* counts_out, void* cuda_stream)
{
    abc_status st;
    if ((st = check_model(1, N_pop, stream)) != ABC_OK) return st;
    if (!valid_mode(mode)) return fail(ABC_ERR_INVALID_ARG, "unknown mode %d", (int)mode);
    if (B > 0 && (!theta || !state_in || !sample_index || !day || !state_out))
        return fail(ABC_ERR_INVALID_ARG, "NULL device buffer");
    if (B == 0) return ok();
    const abcgb::ModelParams p = make_params(nullptr, 1, N_pop, seed, stream, nullptr);
    abcgb::StepArgs a;
    a.theta = theta;
    a.state_in = state_in;
    a.sample_index = sample_index;
    a.day = day;
    a.B = B;
    a.state_out = state_out;
    a.counts_out = counts_out;
    if (injected("launch")) return fail(ABC_ERR_CUDA, "kernel launch failed (injected)");
    CUDA_TRY(abcgb::launch_step(p, a, kernel_mode(mode), (cudaStream_t)cuda_stream), "abc_step_kernel launch");
    return ok();
}

abc_status abc_project(const float* theta, const uint64_t* sample_index, uint64_t B, const int32_t* init_ard,
                       int32_t T, int64_t N_pop, uint64_t seed, uint32_t stream, abc_mode mode,
                       const double* quantiles, int32_t n_q, float* bands_out, void* cuda_stream)
{
    abc_status st;
    if ((st = check_model(T, N_pop, stream)) != ABC_OK) return st;
    if (!valid_mode(mode)) return fail(ABC_ERR_INVALID_ARG, "unknown mode %d", (int)mode);
    if ((st = check_initial(init_ard, N_pop)) != ABC_OK) return st;
    if (B < 1 || B > ABC_PROJECT_MAX_B) return fail(ABC_ERR_INVALID_ARG, "B must be in [1, %d]", ABC_PROJECT_MAX_B);
    if (!theta || !sample_index || !bands_out || !quantiles || n_q < 1 || n_q > 1024)
        return fail(ABC_ERR_INVALID_ARG, "NULL buffer or n_q outside [1, 1024]");
    std::vector<float> qpos((size_t)n_q);
    for (int32_t k = 0; k < n_q; ++k) {
        if (!(quantiles[k] >= 0.0 && quantiles[k] <= 1.0)) return fail(ABC_ERR_INVALID_ARG, "quantile outside [0, 1]");
        qpos[k] = (float)std::floor(quantiles[k] * (double)(B - 1));
    }
    const abcgb::ModelParams p = make_params(nullptr, T, N_pop, seed, stream, init_ard);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    Scratch sc;
    const size_t traj_bytes = sizeof(int32_t) * 6 * (size_t)(T + 1) * B;
    if ((st = alloc_scratch(sc, traj_bytes + sizeof(float) * n_q, s)) != ABC_OK) return st;
    int32_t* traj = (int32_t*)sc.ptr;
    float* qd = (float*)((char*)sc.ptr + traj_bytes);
    CUDA_TRY(cudaMemcpyAsync(qd, qpos.data(), sizeof(float) * n_q, cudaMemcpyHostToDevice, s), "cudaMemcpyAsync(q)");
    abcgb::SimulateArgs a;
    a.theta = theta;
    a.sample_index = sample_index;
    a.B = B;
    a.traj_out = traj;
    if (injected("launch")) return fail(ABC_ERR_CUDA, "kernel launch failed (injected)");
    CUDA_TRY(abcgb::launch_simulate(p, a, kernel_mode(mode), s), "abc_simulate_kernel launch");
    CUDA_TRY(abcgb::launch_bands(traj, (uint32_t)B, T, qd, n_q, bands_out, s), "band_kernel launch");
    // qpos (host) was staged synchronously enough: wait for the copy before it leaves scope
    CUDA_TRY(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    return ok();
}

abc_status abc_kth_smallest(const double* dist, uint64_t n, uint64_t k, double* eps_out, void* cuda_stream)
{
    if (!dist || !eps_out) return fail(ABC_ERR_INVALID_ARG, "NULL pointer");
    if (k < 1 || k > n) return fail(ABC_ERR_INVALID_ARG, "k = %llu outside [1, n = %llu]", (unsigned long long)k,
                                    (unsigned long long)n);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    abc_status st;
    Scratch sc;
    const size_t bytes = 258 * sizeof(unsigned long long) + sizeof(abcgb::SelectState);
    if ((st = alloc_scratch(sc, bytes, s)) != ABC_OK) return st;
    unsigned long long* hist_d = (unsigned long long*)sc.ptr;
    abcgb::SelectState* st_d = (abcgb::SelectState*)(hist_d + 258);   // 16-byte aligned after the 258 counters
    CUDA_TRY(cudaMemsetAsync(sc.ptr, 0, bytes, s), "cudaMemsetAsync(select scratch)");
    if (injected("launch")) return fail(ABC_ERR_CUDA, "kernel launch failed (injected)");
    CUDA_TRY(abcgb::launch_kth_select(dist, n, k, hist_d, st_d, s), "radix select launch");
    abcgb::SelectState h;
    CUDA_TRY(cudaMemcpyAsync(&h, st_d, sizeof h, cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync(select state)");
    CUDA_TRY(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    // keys that are NaN or carry the sign bit do not order like values
    if (h.bad != 0) return fail(ABC_ERR_INVALID_ARG, "%llu distances are negative, -0 or NaN", h.bad);
    std::memcpy(eps_out, &h.prefix, sizeof h.prefix);
    return ok();
}

abc_status abc_select_below(const double* dist, const float* theta, uint64_t n, double eps, uint64_t first_index,
                            float* theta_out, double* dist_out, uint64_t* idx_out, uint64_t capacity,
                            uint64_t* n_selected, void* cuda_stream)
{
    if (!n_selected) return fail(ABC_ERR_INVALID_ARG, "n_selected is NULL");
    *n_selected = 0;
    if (!(eps >= 0.0)) return fail(ABC_ERR_INVALID_ARG, "eps must be >= 0 and not NaN");
    if (n > 0 && !dist) return fail(ABC_ERR_INVALID_ARG, "dist is NULL");
    if (capacity > 0 && (!dist_out || !idx_out || (theta && !theta_out)))
        return fail(ABC_ERR_INVALID_ARG, "an output buffer is NULL");
    if (n > ~(uint64_t)0 - first_index) return fail(ABC_ERR_INVALID_ARG, "first_index + n overflows");
    if (n == 0) return ok();
    cudaStream_t s = (cudaStream_t)cuda_stream;
    abc_status st;
    Scratch sc;
    if ((st = alloc_scratch(sc, sizeof(unsigned long long), s)) != ABC_OK) return st;
    CUDA_TRY(cudaMemsetAsync(sc.ptr, 0, sizeof(unsigned long long), s), "cudaMemsetAsync(count)");
    abcgb::SelectArgs a;
    a.dist = dist;
    a.theta = theta;
    a.n = n;
    a.first_index = first_index;
    a.eps = eps;
    a.eps_key = nullptr;
    a.theta_out = theta ? theta_out : nullptr;
    a.dist_out = dist_out;
    a.idx_out = idx_out;
    a.capacity = capacity;
    a.count = (unsigned long long*)sc.ptr;
    if (injected("launch")) return fail(ABC_ERR_CUDA, "kernel launch failed (injected)");
    CUDA_TRY(abcgb::launch_select_below(a, s), "select_below launch");
    unsigned long long count = 0;
    CUDA_TRY(cudaMemcpyAsync(&count, sc.ptr, sizeof count, cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync(count)");
    CUDA_TRY(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    *n_selected = count;
    if (count > capacity)
        return fail(ABC_ERR_CAPACITY, "%llu samples accepted, capacity %llu", count, (unsigned long long)capacity);
    return ok();
}

abc_status abc_sample_quantile(const abc_prior_box* prior, const int32_t* observed, int32_t T, int64_t N_pop,
                               uint64_t n_samples, uint64_t k, uint64_t seed, uint32_t stream, abc_mode mode,
                               uint64_t first_index, float* theta_out, double* dist_out, uint64_t* idx_out,
                               uint64_t capacity, double* eps_out, uint64_t* n_accepted, void* cuda_stream)
{
    abc_status st;
    if ((st = check_prior(prior)) != ABC_OK) return st;
    if ((st = check_model(T, N_pop, stream)) != ABC_OK) return st;
    if (!valid_mode(mode)) return fail(ABC_ERR_INVALID_ARG, "unknown mode %d", (int)mode);
    if (!eps_out || !n_accepted) return fail(ABC_ERR_INVALID_ARG, "eps_out or n_accepted is NULL");
    *n_accepted = 0;
    if (k < 1 || k > n_samples)
        return fail(ABC_ERR_INVALID_ARG, "k = %llu outside [1, n_samples = %llu]", (unsigned long long)k,
                    (unsigned long long)n_samples);
    if (capacity > 0 && (!theta_out || !dist_out || !idx_out))
        return fail(ABC_ERR_INVALID_ARG, "output buffers are NULL");
    if (n_samples > ~(uint64_t)0 - first_index)
        return fail(ABC_ERR_INVALID_ARG, "first_index + n_samples overflows");
    if (n_samples > (uint64_t)1 << 40) return fail(ABC_ERR_INVALID_ARG, "n_samples above 2^40");
    std::vector<int4> obs;
    if ((st = pack_observed(observed, T, N_pop, obs)) != ABC_OK) return st;
    const int32_t ard0[3] = {obs[0].x, obs[0].y, obs[0].z};
    const abcgb::ModelParams p = make_params(prior, T, N_pop, seed, stream, ard0);
    cudaStream_t s = (cudaStream_t)cuda_stream;

    // every distance and prior draw: stream-ordered scratch, 40 bytes a sample
    const size_t dist_bytes = ((sizeof(double) * n_samples + 255) / 256) * 256;
    Scratch big;
    if ((st = alloc_scratch(big, dist_bytes + sizeof(float) * 8 * n_samples, s)) != ABC_OK) return st;
    double* dist_d = (double*)big.ptr;
    float* theta_d = (float*)((char*)big.ptr + dist_bytes);
    // the radix select's histogram (258 counters) and state, the accept
    // counter, then the observed series: zeroed and uploaded in one copy
    // from pinned staging
    struct Tail {
        abcgb::SelectState sel;
        unsigned long long count;
    };
    const size_t tail_off = 258 * sizeof(unsigned long long), obs_off = 2112;
    static_assert(258 * sizeof(unsigned long long) + sizeof(Tail) <= 2112, "select scratch overlaps the series");
    SampleScratch* sc = nullptr;
    if ((st = sample_scratch(obs_off + sizeof(int4) * obs.size(), &sc)) != ABC_OK) return st;
    std::memset(sc->host, 0, obs_off);
    std::memcpy((char*)sc->host + obs_off, obs.data(), sizeof(int4) * obs.size());
    unsigned long long* hist_d = (unsigned long long*)sc->dev;
    Tail* tail_d = (Tail*)((char*)sc->dev + tail_off);
    Tail* tail_h = (Tail*)((char*)sc->host + tail_off);
    if (injected("launch")) return fail(ABC_ERR_CUDA, "kernel launch failed (injected)");
    // from here on the pinned staging buffer may be in use by the stream: every
    // error return first waits for the stream so the next call can reuse it
    auto drain = [s](abc_status e) {
        cudaStreamSynchronize(s);
        return e;
    };
    cudaError_t ce = cudaMemcpyAsync(sc->dev, sc->host, obs_off + sizeof(int4) * obs.size(), cudaMemcpyHostToDevice, s);
    if (ce != cudaSuccess) return drain(cuda_fail(ce, "cudaMemcpyAsync(observed, counters)"));
    abcgb::DistanceArgs da;
    da.obs = (const int4*)((char*)sc->dev + obs_off);
    da.first_index = first_index;
    da.n_samples = n_samples;
    da.dist_out = dist_d;
    da.theta_out = theta_d;
    ce = abcgb::launch_distances(p, da, kernel_mode(mode), s);
    if (ce != cudaSuccess) return drain(cuda_fail(ce, "abc_distance_kernel launch"));
    ce = abcgb::launch_kth_select(dist_d, n_samples, k, hist_d, &tail_d->sel, s);
    if (ce != cudaSuccess) return drain(cuda_fail(ce, "radix select launch"));
    abcgb::SelectArgs a;
    a.dist = dist_d;
    a.theta = theta_d;
    a.n = n_samples;
    a.first_index = first_index;
    a.eps = 0.0;
    a.eps_key = &tail_d->sel;
    a.theta_out = theta_out;
    a.dist_out = dist_out;
    a.idx_out = idx_out;
    a.capacity = capacity;
    a.count = &tail_d->count;
    ce = abcgb::launch_select_below(a, s);
    if (ce != cudaSuccess) return drain(cuda_fail(ce, "select_below launch"));
    ce = cudaMemcpyAsync(tail_h, tail_d, sizeof(Tail), cudaMemcpyDeviceToHost, s);
    if (ce != cudaSuccess) return drain(cuda_fail(ce, "cudaMemcpyAsync(select state)"));
    CUDA_TRY(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    // the distances of the model are never NaN or negative
    if (tail_h->sel.bad != 0)
        return fail(ABC_ERR_CUDA, "%llu distances are negative, -0 or NaN", tail_h->sel.bad);
    std::memcpy(eps_out, &tail_h->sel.prefix, sizeof(double));
    const unsigned long long count = tail_h->count;
    *n_accepted = count;
    if (count > capacity)
        return fail(ABC_ERR_CAPACITY, "%llu samples accepted, capacity %llu", count, (unsigned long long)capacity);
    return ok();
}

abc_status abc_sample_noalloc(const abc_prior_box* prior, const int32_t* observed, int32_t T, int64_t N_pop,
                              double eps, uint64_t n_samples, uint64_t seed, uint32_t stream, abc_mode mode,
                              uint64_t first_index, float* theta_out, double* dist_out, uint64_t* idx_out,
                              uint64_t capacity, uint64_t* n_accepted, void* cuda_stream)
{
    abc_status st;
    if ((st = check_prior(prior)) != ABC_OK) return st;
    if ((st = check_model(T, N_pop, stream)) != ABC_OK) return st;
    if (T > ABC_NOALLOC_T_MAX)
        return fail(ABC_ERR_INVALID_ARG, "T = %d exceeds the no-alloc scratch limit of %d days", T,
                    ABC_NOALLOC_T_MAX);
    if (!valid_mode(mode)) return fail(ABC_ERR_INVALID_ARG, "unknown mode %d", (int)mode);
    if (!(eps >= 0.0)) return fail(ABC_ERR_INVALID_ARG, "eps must be >= 0 and not NaN");
    if (!n_accepted) return fail(ABC_ERR_INVALID_ARG, "n_accepted is NULL");
    if (capacity > 0 && (!theta_out || !dist_out || !idx_out))
        return fail(ABC_ERR_INVALID_ARG, "output buffers are NULL");
    if (n_samples > ~(uint64_t)0 - first_index)
        return fail(ABC_ERR_INVALID_ARG, "first_index + n_samples overflows");
    if (!observed) return fail(ABC_ERR_INVALID_ARG, "observed is NULL");
    // the observed series, packed on the stack (no heap allocation either)
    int4 obs[ABC_NOALLOC_T_MAX + 1];
    for (int32_t d = 0; d <= T; ++d) {
        const int32_t A = observed[d], R = observed[(T + 1) + d], D = observed[2 * (T + 1) + d];
        if (A < 0 || R < 0 || D < 0) return fail(ABC_ERR_INVALID_ARG, "negative observed count on day %d", d);
        obs[d] = make_int4(A, R, D, 0);
    }
    const int32_t ard0[3] = {obs[0].x, obs[0].y, obs[0].z};
    if ((st = check_initial(ard0, N_pop)) != ABC_OK) return st;
    *n_accepted = 0;
    g_last_sim_days = 0;
    if (n_samples == 0) return ok();

    void* base = nullptr;
    if ((st = noalloc_scratch(&base)) != ABC_OK) return st;
    unsigned long long* count_d = (unsigned long long*)base;
    int4* obs_d = (int4*)((char*)base + 256);
    const abcgb::ModelParams p = make_params(prior, T, N_pop, seed, stream, ard0);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    CUDA_TRY(cudaMemcpyAsync(obs_d, obs, sizeof(int4) * (size_t)(T + 1), cudaMemcpyHostToDevice, s),
             "cudaMemcpyAsync(observed)");
    CUDA_TRY(cudaMemsetAsync(count_d, 0, 3 * sizeof(unsigned long long), s), "cudaMemsetAsync(counters)");
    abcgb::RejectArgs a;
    a.obs = obs_d;
    a.first_index = first_index;
    a.n_samples = n_samples;
    a.acc_max = acc_threshold(eps);
    a.count = count_d;
    a.next = count_d + 1;
    a.sim_days = count_d + 2;
    a.capacity = capacity;
    a.theta_out = theta_out;
    a.dist_out = dist_out;
    a.idx_out = idx_out;
    CUDA_TRY(abcgb::launch_reject(p, a, kernel_mode(mode), s, nullptr), "abc_reject_kernel launch");
    unsigned long long counters[3] = {0, 0, 0};
    CUDA_TRY(cudaMemcpyAsync(counters, count_d, sizeof counters, cudaMemcpyDeviceToHost, s),
             "cudaMemcpyAsync(counters)");
    CUDA_TRY(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    g_last_sim_days = counters[2];
    *n_accepted = counters[0];
    if (counters[0] > capacity)
        return fail(ABC_ERR_CAPACITY, "%llu samples accepted, capacity %llu", counters[0],
                    (unsigned long long)capacity);
    return ok();
}

const char* abc_strerror(abc_status status)
{
    switch (status) {
    case ABC_OK: return "ok";
    case ABC_ERR_INVALID_ARG: return "invalid argument";
    case ABC_ERR_CAPACITY: return "more accepted samples than the output capacity";
    case ABC_ERR_CUDA: return "CUDA error";
    case ABC_ERR_TIMEOUT: return "device wait timed out";
    case ABC_ERR_NOMEM: return "device memory allocation failed";
    }
    return "unknown status";
}

const char* abc_last_error(void) { return g_last_error.c_str(); }

uint64_t abc_last_simulated_days(void) { return g_last_sim_days; }

int abc_version(void) { return 100; }

}  // extern "C"
