// elm_hidden_noalloc: the tensor-core hidden layer with every byte of
// scratch taken from a fixed device array compiled into this library, for
// callers that are not allowed to allocate device memory themselves or
// through the library (see include/elm.h).
#include <mutex>

#include "elm_internal.cuh"

namespace {

// The scratch array: one copy per device that loads this library, held
// until the process exits.  Host code must not use its name as an address;
// the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) char elm_noalloc_scratch[ELM_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 128;
std::mutex g_mu;
char *g_base[kMaxDevices] = {};
unsigned long long g_ctx_id[kMaxDevices] = {};

// Unique id of the current CUDA context (never reused within a process),
// through the driver entry point the runtime exposes; 0 if unavailable.
unsigned long long current_context_id() {
    typedef CUresult (*PFN_get)(CUcontext *);
    typedef CUresult (*PFN_id)(CUcontext, unsigned long long *);
    static PFN_get get = nullptr;
    static PFN_id id = nullptr;
    static bool tried = false;
    if (!tried) {
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess && q == cudaDriverEntryPointSuccess)
            get = (PFN_get)p;
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            id = (PFN_id)p;
        cudaGetLastError();
        tried = true;
    }
    CUcontext c = nullptr;
    unsigned long long v = 0;
    if (!get || !id || get(&c) != CUDA_SUCCESS || !c || id(c, &v) != CUDA_SUCCESS) return 0;
    return v;
}

// Device address of the scratch array in the current context.  It is
// looked up with cudaGetSymbolAddress the first time a device is used, and
// again whenever that device's context has changed since (after
// cudaDeviceReset the module, and so the array, is loaded anew).
char *scratch_base(int dev) {
    if (dev < 0 || dev >= kMaxDevices) throw ElmError(ELM_ERR_UNSUPPORTED, "device ordinal too large");
    std::lock_guard<std::mutex> lk(g_mu);
    const unsigned long long cid = current_context_id();
    if (!g_base[dev] || cid == 0 || cid != g_ctx_id[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, elm_noalloc_scratch);
        if (e != cudaSuccess || !p)
            throw ElmError(ELM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") +
                                             cudaGetErrorString(e));
        g_base[dev] = (char *)p;
        g_ctx_id[dev] = cid;
    }
    return g_base[dev];
}

// Device memory of device `dev` (or managed memory).
bool device_ptr(const void *p, int dev) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

void carve(Arena &ar, int64_t N, int64_t n, int64_t L, elm::OzHidWs *hw,
           __nv_bfloat16 **planes, double **hs, int **err) {
    *hw = elm::oz_hid_carve(ar, N, n, L, 0);
    *planes = (__nv_bfloat16 *)ar.take<char>(elm::oz_gram_planes_bytes(N, L, 0));
    *hs = ar.take<double>(elm::oz_pad(L, 128));
    *err = ar.take<int>(1);
}

}  // namespace

extern "C" int elm_hidden_noalloc_bytes(int64_t N, int64_t n, int64_t L, int64_t *bytes) {
    if (!bytes || N < 1 || n < 1 || L < 1) return ELM_ERR_ARG;
    Arena m;
    elm::OzHidWs hw;
    __nv_bfloat16 *planes;
    double *hs;
    int *err;
    carve(m, N, n, L, &hw, &planes, &hs, &err);
    *bytes = (int64_t)m.used;
    return ELM_OK;
}

extern "C" int elm_hidden_noalloc(const void *X, int x_dtype, int64_t N, int64_t n, int64_t ldx,
                                  const double *W, int64_t ldw, const double *b, const double *a,
                                  int64_t L, int act, double *Ht, int64_t ldh, void *stream) {
    try {
        if (N < 1 || n < 1 || L < 1 || ldx < n || ldw < L || ldh < N) return ELM_ERR_ARG;
        if (L > ELM_MAX_L) return ELM_ERR_ARG;
        if (x_dtype != ELM_F32 && x_dtype != ELM_F64) return ELM_ERR_ARG;
        if (act != ELM_ACT_SIGMOID && act != ELM_ACT_TANH) return ELM_ERR_ARG;
        if (!X || !W || !b || !Ht) return ELM_ERR_ARG;
        // everything runs on the current device: operands and stream must be its own
        int dev = 0;
        ELM_CUDA(cudaGetDevice(&dev));
        if (!device_ptr(X, dev) || !device_ptr(W, dev) || !device_ptr(b, dev) ||
            !device_ptr(Ht, dev) || (a && !device_ptr(a, dev)))
            return ELM_ERR_ARG;
        int sdev = dev;
        ELM_CUDA(cudaStreamGetDevice((cudaStream_t)stream, &sdev));
        if (sdev != dev) return ELM_ERR_ARG;
        Arena m;
        elm::OzHidWs hw;
        __nv_bfloat16 *planes;
        double *hs;
        int *err;
        carve(m, N, n, L, &hw, &planes, &hs, &err);
        if (m.used > (size_t)ELM_NOALLOC_SCRATCH_BYTES) return ELM_ERR_UNSUPPORTED;
        Arena ar;
        ar.base = scratch_base(dev);
        ar.cap = ELM_NOALLOC_SCRATCH_BYTES;
        carve(ar, N, n, L, &hw, &planes, &hs, &err);
        cudaStream_t s = (cudaStream_t)stream;
        // the array keeps the previous call's contents: the error flag must
        // start at zero; every other region is fully rewritten by the kernels
        ELM_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
        elm::oz_hidden(s, hw, X, x_dtype, N, n, ldx, W, ldw, b, a, act, L, 0, planes, hs, Ht,
                       ldh, err);
        int terr = 0;
        ELM_CUDA(cudaMemcpyAsync(&terr, err, sizeof terr, cudaMemcpyDeviceToHost, s));
        ELM_CUDA(cudaStreamSynchronize(s));
        return terr ? ELM_ERR_TIMEOUT : ELM_OK;
    } catch (const ElmError &e) {
        return e.status;
    } catch (...) {
        return ELM_ERR_CUDA;
    }
}
