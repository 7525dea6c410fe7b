// aahrt_forward_noalloc: the forward transform for callers that must not
// allocate device memory during the call.
//
// Some callers cannot call cudaMalloc where they run the transform: code
// under an external device-memory manager that owns the whole heap (a raw
// allocation would fail or fragment its pool), or latency-critical loops
// that forbid allocation and freeing on their hot path.  aahrt_forward
// itself runs on the plan's workspace, but that workspace is one per plan;
// this entry point instead takes its scratch (the model and data spectra and
// the slice kernels' work counter) from one array of fixed size in device
// memory, and allocates nothing.
//
// The array is a file-scope __device__ variable, so every GPU that holds it
// keeps it until the process exits.  With lazy module loading the array is
// committed when this file's module is first loaded on a device; plan
// creation (aahrt_plan_create, aahrt_plan_create_batched) does that, with the
// plan's device current, and looks the array's address up with
// cudaGetSymbolAddress.  Host code cannot use the array's name as a device
// address, so the address of each device is cached and every plan creation
// refreshes it (after a cudaDeviceReset, old plans are invalid anyway and a
// new plan brings a valid address).  The transform call itself therefore
// neither loads a module nor commits memory.
// All calls share the array and it keeps the last call's contents; the work
// counter is cleared on every call and the spectra are fully overwritten.
// Calls whose kernels overlap on the GPU (different streams without
// ordering, or several host threads) race on the array: serialise them.
#include <mutex>
#include <vector>

#include "internal.cuh"

namespace aahrt {

static __device__ __align__(256) unsigned char g_noalloc_scratch[AAHRT_NOALLOC_SCRATCH_BYTES];

static std::mutex g_noalloc_mu;
static std::vector<void *> g_noalloc_addr;   // per device ordinal

// Looks up the array's address on device `dev` (which must be current) and
// caches it; loads this module there first if module loading is lazy.
int noalloc_prepare(int dev) {
    void *ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr) return cuda_fail(e, "allocation-free scratch array address");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if ((int)g_noalloc_addr.size() <= dev) g_noalloc_addr.resize(dev + 1, nullptr);
    g_noalloc_addr[dev] = ptr;
    return AAHRT_OK;
}

// The cached address of device `dev`, set by plan creation on that device.
static int noalloc_base(int dev, unsigned char **out) {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if ((int)g_noalloc_addr.size() <= dev || !g_noalloc_addr[dev])
        return set_error(AAHRT_ERR_INVALID_ARG,
                         "no allocation-free scratch address for device %d (plan not created "
                         "through aahrt_plan_create)", dev);
    *out = static_cast<unsigned char *>(g_noalloc_addr[dev]);
    return AAHRT_OK;
}

static size_t round256(size_t n) { return (n + 255) & ~size_t(255); }

}  // namespace aahrt

using namespace aahrt;

extern "C" int aahrt_forward_noalloc(aahrt_plan *plan, const float *m, float *d, void *stream) {
    if (!plan) return set_error(AAHRT_ERR_INVALID_ARG, "plan is NULL");
    Plan &p = *plan->p;
    DeviceGuard g(p.device);
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess || cur != p.device)
        return set_error(AAHRT_ERR_CUDA, "cannot make the plan's device %d current", p.device);
    int rc = AAHRT_OK;
    do {
        if ((rc = check_dev_ptr(m, "m")) || (rc = check_dev_ptr(d, "d"))) break;
        const size_t xbytes = round256((size_t)p.x_len * sizeof(float2));
        const size_t ybytes = round256((size_t)p.y_len * sizeof(float2));
        const size_t need = 256 + xbytes + ybytes;
        if (need > (size_t)AAHRT_NOALLOC_SCRATCH_BYTES) {
            rc = set_error(AAHRT_ERR_UNSUPPORTED,
                           "plan needs %zu bytes of scratch; aahrt_forward_noalloc has %zu "
                           "(use aahrt_forward)", need, (size_t)AAHRT_NOALLOC_SCRATCH_BYTES);
            break;
        }
        unsigned char *base = nullptr;
        if ((rc = noalloc_base(p.device, &base))) break;
        int *counter = reinterpret_cast<int *>(base);
        float2 *X = reinterpret_cast<float2 *>(base + 256);
        float2 *Y = reinterpret_cast<float2 *>(base + 256 + xbytes);
        cudaStream_t st = (cudaStream_t)stream;
        cudaError_t e;
        if ((e = launch_r2c(p, true, m, X, st))) { rc = cuda_fail(e, "stretch+FFT launch"); break; }
        if ((e = launch_slice(p, false, X, Y, st, counter))) { rc = cuda_fail(e, "slice launch"); break; }
        // deconvolutive plans: synthesis into the plan's (preallocated)
        // convolution workspace, then the time convolution into d
        float *dsyn = p.nw > 0 ? p.wtmp : d;
        if ((e = launch_c2r(p, false, Y, dsyn, EPI_STORE, nullptr, FistaArgs{}, st))) {
            rc = cuda_fail(e, "inverse FFT+unstretch launch");
            break;
        }
        if (p.nw > 0 && (e = launch_wavelet(p, 0, dsyn, d, nullptr, st, false))) {
            rc = cuda_fail(e, "wavelet convolution launch");
            break;
        }
    } while (0);
    return rc;
}
