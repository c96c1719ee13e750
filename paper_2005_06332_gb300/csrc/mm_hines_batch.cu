// mm_hines_batch.cu -- a standalone batched Hines solve on the device.
//
// Algorithm 1 (Sec. 2) exactly as the paper states it, for many independent
// trees at once: one thread per tree walks the backward sweep (leaves to
// root over parent[]) and the forward substitution.  Inputs are const; the
// eliminated diagonal lives in a scratch array and the rhs is worked on in
// the output array.  Device pointers in and out.
#include <cuda_runtime.h>
#include <stdint.h>

#include "mm.h"

// Scratch of mm_hines_solve_noalloc: a fixed device array in this library
// image, so that the call never allocates.  The first 256 bytes hold the
// status word, the rest the eliminated diagonal (MM_NOALLOC_MAX_COMPS doubles,
// 8 MiB).  Every GPU that loads the library holds it until the process ends.
#define MM_NOALLOC_MAX_COMPS (1 << 20)
static __device__ __align__(256) double g_noalloc_scratch[32 + MM_NOALLOC_MAX_COMPS];

namespace {

// status word: 0 = ok, 1 = a tree violates parent[0] = -1, 0 <= parent[i] < i,
// or its entry range tree_offset[t] .. tree_offset[t+1]-1 is not inside
// [0, n_comp) (such a tree is skipped before any of its entries is touched)
__global__ void hines_batch_kernel(int32_t n_trees, int64_t n_comp, const int64_t *__restrict__ off,
                                   const int32_t *__restrict__ parent, const double *__restrict__ a,
                                   const double *__restrict__ b, const double *__restrict__ c,
                                   const double *__restrict__ rhs, double *__restrict__ x,
                                   double *__restrict__ work, int *__restrict__ status)
{
    for (int32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < n_trees; t += gridDim.x * blockDim.x) {
        const int64_t base = off[t], end = off[t + 1];
        if (base < 0 || end < base || end > n_comp) {
            atomicOr(status, 1);
            continue;
        }
        const int64_t n = end - base;
        if (n == 0) continue;
        const int32_t *p = parent + base;
        bool ok = p[0] == -1;
        for (int64_t i = 1; ok && i < n; ++i) ok = p[i] >= 0 && p[i] < i;
        if (!ok) {
            atomicOr(status, 1);
            continue;
        }
        double *w = work + base;
        double *r = x + base;
        for (int64_t i = 0; i < n; ++i) {
            w[i] = b[base + i];
            r[i] = rhs[base + i];
        }
        // backward sweep, leaves to root
        for (int64_t i = n - 1; i >= 1; --i) {
            const double factor = a[base + i] / w[i];
            w[p[i]] -= factor * c[base + i];
            r[p[i]] -= factor * r[i];
        }
        r[0] /= w[0];
        // forward sweep, root to leaves
        for (int64_t i = 1; i < n; ++i) {
            r[i] -= c[base + i] * r[p[i]];
            r[i] /= w[i];
        }
    }
}

mm_status run_batch(int32_t n_trees, int64_t n_comp, const int64_t *off, const int32_t *parent, const double *a,
                    const double *b, const double *c, const double *rhs, double *x, double *work, int *status,
                    cudaStream_t s)
{
    if (cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess) return MM_ECUDA;
    if (n_trees > 0 && n_comp > 0) {
        const int threads = 128;
        int blocks = (int)((n_trees + threads - 1) / threads);
        if (blocks > 152 * 16) blocks = 152 * 16;
        hines_batch_kernel<<<blocks, threads, 0, s>>>(n_trees, n_comp, off, parent, a, b, c, rhs, x, work, status);
        if (cudaGetLastError() != cudaSuccess) return MM_ECUDA;
    }
    int h = 0;
    if (cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return MM_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return MM_ECUDA;
    return h ? MM_EINVAL : MM_OK;
}

bool args_ok(int32_t n_trees, int64_t n_comp, const int64_t *off, const int32_t *parent, const double *a,
             const double *b, const double *c, const double *rhs, double *x)
{
    if (n_trees < 0 || n_comp < 0) return false;
    if (n_trees > 0 && !off) return false;
    if (n_comp > 0 && (!parent || !a || !b || !c || !rhs || !x)) return false;
    return true;
}

}  // namespace

extern "C" mm_status mm_hines_solve(int32_t n_trees, int64_t n_comp, const int64_t *tree_offset,
                                    const int32_t *parent, const double *a, const double *b, const double *c,
                                    const double *rhs, double *x, void *cuda_stream)
{
    if (!args_ok(n_trees, n_comp, tree_offset, parent, a, b, c, rhs, x)) return MM_EINVAL;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // scratch: the eliminated diagonal, then the status word
    const size_t bytes = (size_t)(n_comp > 0 ? n_comp : 1) * sizeof(double) + 256;
    void *scratch = nullptr;
    if (cudaMalloc(&scratch, bytes) != cudaSuccess) {
        cudaGetLastError();
        return MM_ENOMEM;
    }
    double *work = (double *)scratch;
    int *status = (int *)((char *)scratch + bytes - 256);
    const mm_status st = run_batch(n_trees, n_comp, tree_offset, parent, a, b, c, rhs, x, work, status, s);
    cudaFree(scratch);
    return st;
}

// The device address of g_noalloc_scratch is looked up on every call, with
// the caller's device current: in host code the array's name is only a
// host-side stand-in, and a cached address could outlive the module it
// points into (a cudaDeviceReset reloads it).  The lookup allocates nothing.
extern "C" mm_status mm_hines_solve_noalloc(int32_t n_trees, int64_t n_comp, const int64_t *tree_offset,
                                            const int32_t *parent, const double *a, const double *b,
                                            const double *c, const double *rhs, double *x, void *cuda_stream)
{
    if (!args_ok(n_trees, n_comp, tree_offset, parent, a, b, c, rhs, x)) return MM_EINVAL;
    if (n_comp > MM_NOALLOC_MAX_COMPS) return MM_EINVAL;
    void *base = nullptr;
    if (cudaGetSymbolAddress(&base, g_noalloc_scratch) != cudaSuccess || !base) {
        cudaGetLastError();
        return MM_ECUDA;
    }
    int *status = (int *)base;                       // cleared by run_batch before the kernel
    double *work = (double *)((char *)base + 256);   // fully written before it is read
    return run_batch(n_trees, n_comp, tree_offset, parent, a, b, c, rhs, x, work, status,
                     (cudaStream_t)cuda_stream);
}
