// fs_edges.cu - segment edges given as frequencies in device memory, and the
// check of a caller's frequency grid.
//
// Sec. II.B: with the number of segments fixed, bin k belongs to segment p iff
// e_p <= f_k < e_{p+1}, the last segment closed at e_{N_p}.  The fused kernels
// work on bin indices, so one small kernel turns the caller's N_p + 1 edge
// frequencies into segment starts before every evaluation:
//   start[p]   = #{k : f_k <  e_p}   (p < N_p)
//   start[N_p] = #{k : f_k <= e_{N_p}}
// and segment p is the bins [start[p], start[p+1]).  The conversion runs on the
// stream, inside any captured graph, so each evaluation reads the edges the
// caller's buffer holds when it runs, and nothing waits on the host.
//
// Edges that are not finite or decrease cannot be refused synchronously
// without a host wait; the kernel then writes empty segments, clears the
// validity word start[N_p + 1] (the solve kernel turns that into F = NaN) and
// sets bit 0 of a sticky device flag word.
#include "fs_internal.h"
#include "fs_device.cuh"

namespace fs {

// Number of bins with f_k < x (inclusive = false) or f_k <= x (inclusive =
// true), by bisection on the exact predicate: f_k increases with k, and bin_freq
// rounds as every other kernel does.
__device__ int64_t bins_below(const Grid& g, double x, bool inclusive) {
    int64_t lo = 0, hi = g.n;   // answer in [lo, hi]
    while (lo < hi) {           // at most 41 rounds for n <= 2^40
        const int64_t mid = lo + (hi - lo) / 2;
        const double f = bin_freq(g, mid);
        const bool past = inclusive ? f > x : f >= x;
        if (past) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

__global__ void edges_kernel(Grid g, const double* __restrict__ e, int Np, int64_t* starts, int* flags) {
    bool ok = true;
    for (int p = threadIdx.x; p <= Np; p += blockDim.x) {
        const double x = e[p];
        if (!isfinite(x) || (p > 0 && !(e[p - 1] <= x))) ok = false;
    }
    ok = __syncthreads_and(ok) != 0;
    for (int p = threadIdx.x; p <= Np; p += blockDim.x)
        starts[p] = ok ? bins_below(g, e[p], p == Np) : 0;
    if (threadIdx.x == 0) {
        starts[Np + 1] = ok ? 1 : 0;
        if (!ok && flags) atomicOr(flags, kFlagBadEdges);
    }
}

cudaError_t launch_edges(const Grid& g, const double* edges_hz, int Np, int64_t* starts, int* flags,
                         cudaStream_t s) {
    edges_kernel<<<1, 256, 0, s>>>(g, edges_hz, Np, starts, flags);
    return cudaGetLastError();
}

// A caller's grid agrees with f_k = f_min + k df when every value is within 4
// units in the last place of f_k (rounding of another evaluation order).
__global__ void grid_check_kernel(Grid g, const double* __restrict__ fg, int* flags) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool bad = false;
    if (k < g.n) {
        const double f = bin_freq(g, k);
        bad = !(fabs(fg[k] - f) <= 8.881784197001252e-16 * f);   // 4 * 2^-52
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flags, kFlagBadGrid);
}

cudaError_t launch_grid_check(const Grid& g, const double* f_grid, int* flags, cudaStream_t s) {
    const int threads = 256;
    grid_check_kernel<<<(unsigned)((g.n + threads - 1) / threads), threads, 0, s>>>(g, f_grid, flags);
    return cudaGetLastError();
}

}  // namespace fs
