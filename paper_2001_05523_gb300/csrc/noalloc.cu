// Allocation-free apply: y = A x with the work vectors in a fixed,
// library-owned device array instead of memory allocated per operator.
//
// h2bem_apply allocates its device work vectors with cudaMalloc on its first
// call and whenever nrhs grows.  A caller that cannot let a library allocate at
// apply time (one whose device memory is all handed out by its own pool
// allocator, so a cudaMalloc here would fail or force the pool to release
// memory; one that must not trigger the implicit device synchronisation a
// cudaMalloc/cudaFree may cause inside a latency-critical loop) uses this entry
// point instead.  It calls no cudaMalloc, cudaFree or allocating library
// routine: its scratch space is the file-scope array below, which every GPU
// that loads the library holds from module load until the process exits.
#include <cstdio>
#include <mutex>

#include "../../include/h2bem.h"
#include "internal.h"

namespace {

constexpr size_t kScratchBytes = size_t(64) << 20;  // 64 MiB per device
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mutex;
unsigned char* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_scratch on the current device.  In host code the name
// g_scratch is only a host-side stand-in, so the address is looked up once per
// device (with that device current) and cached.
int scratch_address(unsigned char** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        char msg[160];
        snprintf(msg, sizeof msg, "apply_noalloc: no usable current device (%s)", cudaGetErrorString(e));
        return h2::set_error(H2BEM_ERR_CUDA, msg);
    }
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            char msg[160];
            snprintf(msg, sizeof msg, "apply_noalloc: cudaGetSymbolAddress failed (%s)", cudaGetErrorString(e));
            return h2::set_error(H2BEM_ERR_CUDA, msg);
        }
        g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_scratch_ptr[dev];
    return H2BEM_OK;
}

// Device (or managed) memory of the current device: the scratch array used is
// the current device's, so buffers of another GPU are refused.
bool on_device(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

}  // namespace

extern "C" int h2bem_apply_noalloc(h2bem_op* op, const double* x, int64_t ldx, int nrhs, double* y, int64_t ldy,
                                   void* stream) {
    if (!op || !x || !y) return h2::set_error(H2BEM_ERR_ARG, "apply_noalloc: NULL argument");
    const int64_t n = h2::op_size(op);
    if (nrhs < 1 || nrhs > 64) return h2::set_error(H2BEM_ERR_ARG, "apply_noalloc: nrhs must be in 1..64");
    if (ldx < n || ldy < n) return h2::set_error(H2BEM_ERR_ARG, "apply_noalloc: leading dimensions must be >= n");
    {
        const char* xb = (const char*)x;
        const char* xe = (const char*)(x + (nrhs - 1) * ldx + n);
        const char* yb = (const char*)y;
        const char* ye = (const char*)(y + (nrhs - 1) * ldy + n);
        if (xb < ye && yb < xe) return h2::set_error(H2BEM_ERR_ARG, "apply_noalloc: x and y overlap");
    }
    if (!on_device(x) || !on_device(y))
        return h2::set_error(H2BEM_ERR_ARG, "apply_noalloc: x and y must be device memory of the current device");
    const int chunk = nrhs < 16 ? nrhs : 16;
    const int NR = chunk <= 1 ? 1 : chunk <= 4 ? 4 : chunk <= 8 ? 8 : 16;
    const size_t need = h2::work_bytes(op, NR);
    if (need > kScratchBytes) {
        char msg[200];
        snprintf(msg, sizeof msg,
                 "apply_noalloc: this operator needs %zu bytes of work space for %d right-hand sides per pass, "
                 "more than the fixed %zu bytes; use h2bem_apply",
                 need, NR, kScratchBytes);
        return h2::set_error(H2BEM_ERR_ARG, msg);
    }
    unsigned char* work = nullptr;
    int rc = scratch_address(&work);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    for (int c0 = 0; c0 < nrhs; c0 += 16) {
        const int nr = nrhs - c0 < 16 ? nrhs - c0 : 16;
        rc = h2::apply_with_work(op, x + c0 * ldx, ldx, nr, y + c0 * ldy, ldy, s, work);
        if (rc) return rc;
    }
    return H2BEM_OK;
}
