// Strongly connected components of the arena and their topological levels,
// for SCC-ordered solving (the closing remark of Sec. 6: partition the arena
// into strongly connected components and process them in topological order).
//
// The least fixpoint at a vertex depends only on the vertices it reaches.
// Give every component the level 0 if no edge leaves it, else one more than
// the highest level its edges lead to; then the vertices of level l depend
// only on levels <= l, and solving level 0, 1, ... in turn -- each level
// with the values of the lower ones final -- gives the least fixpoint.
//
// The components are found on the device by repeating, on the vertices not
// yet assigned:
//   trim     a vertex with no unassigned successor or no unassigned
//            predecessor is a component by itself (repeated to exhaustion);
//   colour   every vertex takes the largest id among the vertices that reach
//            it (max-label propagation over the edges);
//   close    a vertex whose colour is its own id is a root; the vertices of
//            that colour that reach the root (backward propagation from it
//            within the colour) are exactly the root's component.
// Levels then come from Kahn's rounds over the condensation: components
// with no edge to another component are level 0; removing a level frees the
// components whose last outgoing edges led into it.  After MAX_LEVELS rounds
// the remaining components share one last level (solving components of
// several levels together is still correct, only less ordered).
#include <cuda_runtime.h>

#include <algorithm>

#include "eg_device.cuh"
#include "eg_internal.h"

namespace eg {

constexpr int SCC_THREADS = 256;
constexpr int MAX_LEVELS = 4096;

static int grid_for(long long items, int sms) {
    return (int)std::max<long long>(1, std::min<long long>((items + SCC_THREADS - 1) / SCC_THREADS, (long long)sms * 8));
}

// Counts of unassigned successors and predecessors of every unassigned vertex.
__global__ void k_scc_counts(DevArena A, const int *comp, int *outc, int *inc) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < A.n; v += gridDim.x * blockDim.x) {
        if (comp[v] >= 0) continue;
        int o = 0, i = 0;
        for (int e = A.row_ptr[v]; e < A.row_ptr[v + 1]; ++e) o += comp[A.col[e]] < 0 && A.col[e] != v;
        for (int e = A.rrow_ptr[v]; e < A.rrow_ptr[v + 1]; ++e) {
            const int p = (int)(A.rcol[e] & 0x7fffffffu);
            i += comp[p] < 0 && p != v;
        }
        outc[v] = o;
        inc[v] = i;
    }
}

// One trimming pass: an unassigned vertex without unassigned successors or
// predecessors (self-loops aside) becomes its own component; its neighbours'
// counts drop.  changed[0] is set when a vertex was trimmed.
__global__ void k_scc_trim(DevArena A, int *comp, int *outc, int *inc, unsigned *changed) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < A.n; v += gridDim.x * blockDim.x) {
        if (comp[v] >= 0) continue;
        if (ld_cg(outc + v) > 0 && ld_cg(inc + v) > 0) continue;
        if (atomicCAS(comp + v, -1, v) != -1) continue;
        for (int e = A.row_ptr[v]; e < A.row_ptr[v + 1]; ++e) {
            const int u = A.col[e];
            if (u != v) atomicSub(inc + u, 1);
        }
        for (int e = A.rrow_ptr[v]; e < A.rrow_ptr[v + 1]; ++e) {
            const int p = (int)(A.rcol[e] & 0x7fffffffu);
            if (p != v) atomicSub(outc + p, 1);
        }
        *changed = 1;
    }
}

__global__ void k_scc_color_init(int n, const int *comp, int *color) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        color[v] = comp[v] >= 0 ? -1 : v;
}

// Max-label propagation along edges between unassigned vertices.
__global__ void k_scc_color(DevArena A, const int *comp, int *color, unsigned *changed) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < A.n; v += gridDim.x * blockDim.x) {
        if (comp[v] >= 0) continue;
        const int c = ld_cg(color + v);
        for (int e = A.row_ptr[v]; e < A.row_ptr[v + 1]; ++e) {
            const int u = A.col[e];
            if (comp[u] < 0 && ld_cg(color + u) < c && atomicMax(color + u, c) < c) *changed = 1;
        }
    }
}

// Roots (colour = own id) seed their components.
__global__ void k_scc_roots(int n, int *comp, const int *color, int *mark) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        mark[v] = comp[v] < 0 && color[v] == v ? v : -1;
}

// Backward closure within a colour: an unmarked vertex with a successor of
// its colour already marked joins that component.
__global__ void k_scc_close(DevArena A, const int *comp, const int *color, int *mark, unsigned *changed) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < A.n; v += gridDim.x * blockDim.x) {
        if (comp[v] >= 0 || ld_cg(mark + v) >= 0) continue;
        const int c = color[v];
        for (int e = A.row_ptr[v]; e < A.row_ptr[v + 1]; ++e) {
            const int u = A.col[e];
            if (comp[u] < 0 && color[u] == c && ld_cg(mark + u) == c) {
                mark[v] = c;
                *changed = 1;
                break;
            }
        }
    }
}

__global__ void k_scc_commit(int n, int *comp, const int *mark) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        if (comp[v] < 0 && mark[v] >= 0) comp[v] = mark[v];
}

// Per component (indexed by its representative id): edges that leave it.
__global__ void k_scc_outdeg(DevArena A, const int *comp, int *cout) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < A.n; v += gridDim.x * blockDim.x) {
        const int c = comp[v];
        int x = 0;
        for (int e = A.row_ptr[v]; e < A.row_ptr[v + 1]; ++e) x += comp[A.col[e]] != c;
        if (x) atomicAdd(cout + c, x);
    }
}

__global__ void k_scc_level0(int n, const int *comp, const int *cout, int *clevel) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        if (comp[v] == v) clevel[v] = cout[v] == 0 ? 0 : -1;
}

// Kahn's round l: every vertex of a level-l component takes its edges out of
// the counts of its predecessors' components; a component whose count
// reaches 0 is level l + 1.
__global__ void k_scc_release(DevArena A, const int *comp, int *cout, int *clevel, int l, unsigned *changed) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < A.n; v += gridDim.x * blockDim.x) {
        const int c = comp[v];
        if (ld_cg(clevel + c) != l) continue;
        for (int e = A.rrow_ptr[v]; e < A.rrow_ptr[v + 1]; ++e) {
            const int pc = comp[(int)(A.rcol[e] & 0x7fffffffu)];
            if (pc == c) continue;
            if (atomicSub(cout + pc, 1) == 1) {
                clevel[pc] = l + 1;
                *changed = 1;
            }
        }
    }
}

__global__ void k_scc_vertex_level(int n, const int *comp, const int *clevel, int last, int *level) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const int l = clevel[comp[v]];
        level[v] = l < 0 ? last : l;
    }
}

// flag[0] = 1 if some vertex has no component yet.
__global__ void k_scc_unassigned(int n, const int *comp, unsigned *flag) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        if (comp[v] < 0) *flag = 1;
}

// out[0] = highest level, out[1] = number of components.
__global__ void k_scc_summary(int n, const int *comp, const int *level, int *out) {
    int lmax = 0, roots = 0;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        lmax = max(lmax, level[v]);
        roots += comp[v] == v;
    }
    for (int d = 16; d; d >>= 1) {
        lmax = max(lmax, __shfl_down_sync(FULL, lmax, d));
        roots += __shfl_down_sync(FULL, roots, d);
    }
    if (lane_id() == 0) {
        atomicMax(out, lmax);
        atomicAdd(out + 1, roots);
    }
}

// Iterates a kernel until it reports no change; returns the passes made.
template <typename F>
static eg_status until_stable(F pass, unsigned *dflag, unsigned *hflag, cudaStream_t s, int &passes) {
    passes = 0;
    for (;;) {
        EG_CUDA_TRY(cudaMemsetAsync(dflag, 0, 4, s));
        pass();
        EG_CUDA_TRY(cudaGetLastError());
        EG_CUDA_TRY(cudaMemcpyAsync(hflag, dflag, 4, cudaMemcpyDeviceToHost, s));
        EG_CUDA_TRY(cudaStreamSynchronize(s));
        ++passes;
        if (!*hflag) return EG_OK;
    }
}

eg_status scc_levels(eg_arena *ar, cudaStream_t s) {
    if (ar->scc_level) return EG_OK;
    const int n = ar->n;
    int sms = 0;
    EG_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ar->device));
    const int g = grid_for(n, sms);
    int *level = nullptr, *comp = nullptr, *tmp = nullptr;
    eg_status rc = EG_OK;
    auto fail = [&](cudaError_t e) {
        set_error("strongly connected components: %s", cudaGetErrorString(e));
        rc = e == cudaErrorMemoryAllocation ? EG_ERR_OOM : EG_ERR_CUDA;
    };
    cudaError_t e = cudaMalloc((void **)&level, (size_t)n * 4);
    if (e == cudaSuccess) e = cudaMalloc((void **)&comp, (size_t)n * 4);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&tmp, (size_t)n * 4 * 4 + 256, s);
    if (e != cudaSuccess) fail(e);
    int *outc = tmp, *inc = tmp + n, *color = tmp + 2 * (size_t)n, *mark = tmp + 3 * (size_t)n;
    unsigned *dflag = tmp ? (unsigned *)(tmp + 4 * (size_t)n) : nullptr;
    unsigned *hflag = (unsigned *)ar->host_ctrl;
    const DevArena A = ar->d;
    int passes = 0, total = 0;
    if (rc == EG_OK && (e = cudaMemsetAsync(comp, 0xff, (size_t)n * 4, s)) != cudaSuccess) fail(e);
    // each outer pass assigns at least the component of the largest
    // unassigned id (its colour is its own id)
    while (rc == EG_OK) {
        k_scc_counts<<<g, SCC_THREADS, 0, s>>>(A, comp, outc, inc);
        if ((rc = until_stable([&] { k_scc_trim<<<g, SCC_THREADS, 0, s>>>(A, comp, outc, inc, dflag); }, dflag,
                               hflag, s, passes)) != EG_OK)
            break;
        total += passes;
        k_scc_color_init<<<g, SCC_THREADS, 0, s>>>(n, comp, color);
        if ((rc = until_stable([&] { k_scc_color<<<g, SCC_THREADS, 0, s>>>(A, comp, color, dflag); }, dflag, hflag,
                               s, passes)) != EG_OK)
            break;
        total += passes;
        k_scc_roots<<<g, SCC_THREADS, 0, s>>>(n, comp, color, mark);
        if ((rc = until_stable([&] { k_scc_close<<<g, SCC_THREADS, 0, s>>>(A, comp, color, mark, dflag); }, dflag,
                               hflag, s, passes)) != EG_OK)
            break;
        total += passes;
        k_scc_commit<<<g, SCC_THREADS, 0, s>>>(n, comp, mark);
        // another outer pass while a vertex has no component
        if ((e = cudaMemsetAsync(dflag, 0, 4, s)) != cudaSuccess) {
            fail(e);
            break;
        }
        k_scc_unassigned<<<g, SCC_THREADS, 0, s>>>(n, comp, dflag);
        if ((e = cudaGetLastError()) != cudaSuccess ||
            (e = cudaMemcpyAsync(hflag, dflag, 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess) {
            fail(e);
            break;
        }
        if (!*hflag) break;
    }
    int nlev = 0, h[2] = {0, 0};
    if (rc == EG_OK) {
        // levels: Kahn's rounds over the condensation
        int *cout = outc, *clevel = inc;
        if ((e = cudaMemsetAsync(cout, 0, (size_t)n * 4, s)) != cudaSuccess ||
            (e = cudaMemsetAsync(clevel, 0xff, (size_t)n * 4, s)) != cudaSuccess) {
            fail(e);
        } else {
            k_scc_outdeg<<<g, SCC_THREADS, 0, s>>>(A, comp, cout);
            k_scc_level0<<<g, SCC_THREADS, 0, s>>>(n, comp, cout, clevel);
            int l = 0;
            for (; l < MAX_LEVELS - 1 && rc == EG_OK; ++l) {
                if ((e = cudaMemsetAsync(dflag, 0, 4, s)) != cudaSuccess) {
                    fail(e);
                    break;
                }
                k_scc_release<<<g, SCC_THREADS, 0, s>>>(A, comp, cout, clevel, l, dflag);
                if ((e = cudaGetLastError()) != cudaSuccess ||
                    (e = cudaMemcpyAsync(hflag, dflag, 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
                    (e = cudaStreamSynchronize(s)) != cudaSuccess) {
                    fail(e);
                    break;
                }
                if (!*hflag) break;
            }
            total += l + 1;
            k_scc_vertex_level<<<g, SCC_THREADS, 0, s>>>(n, comp, clevel, l + 1, level);
            int *dsum = (int *)dflag;
            if (rc == EG_OK && ((e = cudaMemsetAsync(dsum, 0, 8, s)) != cudaSuccess)) fail(e);
            k_scc_summary<<<g, SCC_THREADS, 0, s>>>(n, comp, level, dsum);
            if (rc == EG_OK && ((e = cudaGetLastError()) != cudaSuccess ||
                                (e = cudaMemcpyAsync(h, dsum, 8, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
                                (e = cudaStreamSynchronize(s)) != cudaSuccess))
                fail(e);
            nlev = h[0] + 1;
        }
    }
    if (tmp) cudaFreeAsync(tmp, s);
    if (rc != EG_OK) {
        if (level) cudaFree(level);
        if (comp) cudaFree(comp);
        return rc;
    }
    ar->scc_level = level;
    ar->scc_comp = comp;
    ar->scc_nlevels = nlev;
    ar->scc_count = h[1];
    ar->scc_passes = total;
    return EG_OK;
}

}  // namespace eg
