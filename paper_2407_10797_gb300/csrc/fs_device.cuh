// fs_device.cuh - device helpers shared by the FP64 and mixed-precision kernels.
#pragma once

#include "fs_internal.h"

namespace fs {

__device__ __forceinline__ FreqPowers powers_of(double f) {
    FreqPowers w;
    w.u = rcbrt(f);
    double u2 = w.u * w.u;
    w.g0h = u2 * u2 * w.u;
    w.e19 = pow(kF0Ecc / f, 19.0 / 9.0);
    return w;
}

__device__ __forceinline__ double bin_freq(const Grid& g, int64_t k) {
    // the same two roundings as f_min + (double)k * df without contraction
    return __dadd_rn(g.f_min, __dmul_rn((double)k, g.df));
}

// ---------------------------------------------------------------------------
// Segment helpers (device)
// ---------------------------------------------------------------------------
struct SegView {
    int Np;
    int global;
    const int64_t* edges;
    int64_t lo, hi;   // band [lo, hi] inclusive
    __device__ int seg(int64_t k) const {
        if (!global) return seg_of_bin(k, lo, hi, Np);
        // largest p with edges[p] <= k (edges non-decreasing, k in [edges[0], edges[Np]))
        int a = 0, b = Np;   // invariant: edges[a] <= k < edges[b]
        while (b - a > 1) {
            int m = (a + b) >> 1;
            if (edges[m] <= k) a = m; else b = m;
        }
        return a;
    }
    // first bin of segment p (p = 0..Np)
    __device__ int64_t start(int p) const {
        if (global) return edges[p];
        if (p >= Np) return hi + 1;
        int64_t w = hi - lo;
        if (w == 0) return p == 0 ? lo : hi + 1;
        int64_t num = (int64_t)p * w;
        return lo + (num + Np - 1) / Np;
    }
};

__device__ __forceinline__ SegView seg_view(const Segs& sg, const Particle& P) {
    SegView v;
    v.Np = sg.Np;
    v.global = sg.global;
    v.edges = sg.edges;
    if (sg.global) {
        v.lo = sg.edges[0];
        v.hi = sg.edges[sg.Np] - 1;
    } else {
        v.lo = P.klo;
        v.hi = P.khi;
    }
    return v;
}

// Work item `item` of the persistent kernels' order (every heavy item, then
// the others; the span-list buffer layout is launch_span_lists'): its span
// and particle.  Warp-uniform; false once item is past the last one.
__device__ __forceinline__ bool sched_item(const int* __restrict__ sched, int nspans, int B,
                                           const int* __restrict__ list, int item, int& span, int& b) {
    const int* off_h = sched + nspans;
    const int* nh = sched + 2 * nspans + 4;
    const int* off_l = sched + 3 * nspans + 4;
    const int th = off_h[nspans];
    const bool heavy = item < th;
    const int i = heavy ? item : item - th;
    const int* off = heavy ? off_h : off_l;
    if (i >= off[nspans]) return false;
    // span = the last s with off[s] <= i (off is non-decreasing, off[0] = 0)
    int lo = 0, hi = nspans;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= i) lo = mid;
        else hi = mid;
    }
    span = lo;
    b = list[(int64_t)lo * B + (i - off[lo]) + (heavy ? 0 : nh[lo])];
    return true;
}

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// ---------------------------------------------------------------------------
// 64-bit fixed-point phase (cycles mod 1 in units of 2^-64)
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long to_fixed(double x) {
    double y = x - floor(x);          // [0, 1)
    double a = y * 4294967296.0;
    double hi = floor(a);
    double lo = (a - hi) * 4294967296.0;
    return ((unsigned long long)hi << 32) + (unsigned long long)lo;
}

// Fixed-point fraction of a small value (|x| < 0.5 cycle) without the floor.
__device__ __forceinline__ unsigned long long to_fixed_small(double x) {
    if (!(fabs(x) < 0.5)) return to_fixed(x);
    return (unsigned long long)__double2ll_rn(x * 18446744073709551616.0);
}

// Phase polynomial at integer offset d (exact modulo 2^64).
__device__ __forceinline__ unsigned long long poly_fx(const unsigned long long c[4], long long d) {
    unsigned long long u = (unsigned long long)d;
    return c[0] + u * (c[1] + u * (c[2] + u * c[3]));
}

// ---------------------------------------------------------------------------
// Polynomials in the bin offset (anchored kernels)
// ---------------------------------------------------------------------------
// p <- p * u, truncated at degree KD (u[0] = 0, u of degree NU)
template <int KD, int NU, typename T>
__device__ __forceinline__ void poly_mul_u(T* p, const T* u) {
#pragma unroll
    for (int k = KD; k >= 1; k--) {
        T s = T(0);
#pragma unroll
        for (int j = 1; j <= NU && j <= k; j++) s = fma(u[j], p[k - j], s);
        p[k] = s;
    }
    p[0] = T(0);
}

// Coefficients of sum_{n=0..na} a[n] u(d)^n, truncated at degree KD, by Horner's
// scheme on polynomials (u of degree NU with u[0] = 0).
template <int KD, int NU, typename T>
__device__ __forceinline__ void poly_compose(const T* a, int na, const T* u, T* out) {
    for (int k = 0; k <= KD; k++) out[k] = T(0);
    out[0] = a[na];
    for (int n = na - 1; n >= 0; n--) {
        poly_mul_u<KD, NU, T>(out, u);
        out[0] += a[n];
    }
}

// ---------------------------------------------------------------------------
// Launch helpers (host)
// ---------------------------------------------------------------------------
// Resident CTAs per SM times SMs for a persistent kernel, cached per device.
template <typename K>
inline int persistent_grid(K kernel, int threads, size_t smem, int variant_slot) {
    static int cache[64][4];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    int& v = cache[dev][variant_slot];
    if (v > 0) return v;
    int nsm = 0, per = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem) != cudaSuccess) return 0;
    v = nsm * (per > 0 ? per : 1);
    return v;
}


}  // namespace fs
