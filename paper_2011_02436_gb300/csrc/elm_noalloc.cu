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

// Device address of the scratch array on the current device, resolved
// once per device with that device current.
char *scratch_base(int dev) {
    if (dev < 0 || dev >= kMaxDevices) throw ElmError(ELM_ERR_UNSUPPORTED, "device ordinal too large");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_base[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, elm_noalloc_scratch);
        if (e != cudaSuccess || !p)
            throw ElmError(ELM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") +
                                             cudaGetErrorString(e));
        g_base[dev] = (char *)p;
    }
    return g_base[dev];
}

bool device_ptr(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
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
        if (!device_ptr(X) || !device_ptr(W) || !device_ptr(b) || !device_ptr(Ht) ||
            (a && !device_ptr(a)))
            return ELM_ERR_ARG;
        Arena m;
        elm::OzHidWs hw;
        __nv_bfloat16 *planes;
        double *hs;
        int *err;
        carve(m, N, n, L, &hw, &planes, &hs, &err);
        if (m.used > (size_t)ELM_NOALLOC_SCRATCH_BYTES) return ELM_ERR_UNSUPPORTED;
        int dev = 0;
        ELM_CUDA(cudaGetDevice(&dev));
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
