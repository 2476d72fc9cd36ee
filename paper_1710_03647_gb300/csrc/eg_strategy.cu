// Winning strategy of player 0 (eg_strategy), read off the least EPM that
// eg_solve_credit computes.
#include <cuda_runtime.h>

#include <algorithm>

#include "eg_device.cuh"
#include "eg_internal.h"

// Every player-0 vertex
// with a finite credit moves along its first out-edge (CSR order) that
// attains the credit, f(u) (-) w'(v, u) = f(v).  On every cycle of chosen
// edges f(v_i) >= f(v_{i+1}) - w'_i, so its weight is >= 0, and player-1
// vertices satisfy f(v) >= f(u) (-) w' for every successor: from v the
// strategy never needs more than f(v) energy (Def. "EPM", Sec. 3.1).

namespace eg {

template <typename T>
__global__ void k_strategy(DevArena A, WeightView W, const T *f, int *succ, unsigned long long *missing) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < A.n; v += gridDim.x * blockDim.x) {
        int pick = -1;
        const T fv = f[v];
        const bool p1 = (__ldg(A.owner_bits + (v >> 5)) >> (v & 31)) & 1u;
        if (!p1 && fv != Cred<T>::TOP) {
            const int e1 = __ldg(A.row_ptr + v + 1);
            for (int e = __ldg(A.row_ptr + v); e < e1; ++e) {
                const int u = __ldg(A.col + e);
                if (ominus<T>(f[u], wmap(__ldg(A.w + e), W), W.C) == fv) {
                    pick = u;
                    break;
                }
            }
            if (pick < 0) atomicAdd(missing, 1ull);
        }
        succ[v] = pick;
    }
}

static size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

static int sm_count(int device) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    return sms > 0 ? sms : 1;
}

static bool is_device_ptr(const void *p) {
    cudaPointerAttributes attr{};
    const bool dev = p && cudaPointerGetAttributes(&attr, p) == cudaSuccess &&
                     (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    return dev;
}

static eg_status strategy(eg_arena *ar, int credit_bits, long long scale, long long shift, const void *credits,
                          int32_t *succ_out, cudaStream_t s) {
    if (credit_bits != 32 && credit_bits != 64) {
        set_error("credit_bits must be 32 or 64");
        return EG_ERR_INVALID;
    }
    const long long sa = scale < 0 ? -scale : scale, sh = shift < 0 ? -shift : shift;
    if (sa > (1LL << 30) || sh > (1LL << 61)) {
        set_error("weight map out of range");
        return EG_ERR_INVALID;
    }
    long long C = 0, wmax = 0;
    eg_status rc = compute_bound(ar, scale, shift, &C, &wmax, s);
    if (rc != EG_OK) return rc;
    const size_t n = (size_t)ar->n, cb = n * (credit_bits / 8);
    const bool dev_in = is_device_ptr(credits), dev_out = is_device_ptr(succ_out);
    char *tmp = nullptr;
    const size_t o_succ = align_up(cb), o_miss = o_succ + align_up(n * 4);
    EG_CUDA_TRY(cudaMallocAsync((void **)&tmp, o_miss + 256, s));
    const void *f = credits;
    if (!dev_in) {
        EG_CUDA_TRY(cudaMemcpyAsync(tmp, credits, cb, cudaMemcpyHostToDevice, s));
        f = tmp;
    }
    int *succ = dev_out ? succ_out : (int *)(tmp + o_succ);
    unsigned long long *miss = (unsigned long long *)(tmp + o_miss), hmiss = 0;
    EG_CUDA_TRY(cudaMemsetAsync(miss, 0, 8, s));
    const int blocks = (int)std::min<long long>(((long long)n + 255) / 256, (long long)sm_count(ar->device) * 16);
    const WeightView W{scale, shift, C};
    if (credit_bits == 32) k_strategy<int><<<blocks, 256, 0, s>>>(ar->d, W, (const int *)f, succ, miss);
    else k_strategy<long long><<<blocks, 256, 0, s>>>(ar->d, W, (const long long *)f, succ, miss);
    EG_CUDA_TRY(cudaGetLastError());
    if (!dev_out) EG_CUDA_TRY(cudaMemcpyAsync(succ_out, succ, n * 4, cudaMemcpyDeviceToHost, s));
    EG_CUDA_TRY(cudaMemcpyAsync(&hmiss, miss, 8, cudaMemcpyDeviceToHost, s));
    EG_CUDA_TRY(cudaFreeAsync(tmp, s));
    EG_CUDA_TRY(cudaStreamSynchronize(s));
    if (hmiss) {
        set_error("%llu player-0 credits are attained by no out-edge: not the least EPM of this arena and map",
                  (unsigned long long)hmiss);
        return EG_ERR_INVALID;
    }
    return EG_OK;
}

}  // namespace eg

extern "C" eg_status eg_strategy(eg_arena *arena, int32_t credit_bits, int64_t w_scale, int64_t w_shift,
                                 const void *credits, int32_t *succ_out, void *cuda_stream) {
    eg::clear_error();
    if (!arena || !credits || !succ_out) {
        eg::set_error("arena, credits and succ_out are required");
        return EG_ERR_INVALID;
    }
    try {
        return eg::strategy(arena, credit_bits, w_scale, w_shift, credits, succ_out, (cudaStream_t)cuda_stream);
    } catch (...) {
        eg::set_error("unexpected exception in eg_strategy");
        return EG_ERR_INVALID;
    }
}

