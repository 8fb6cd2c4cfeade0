// scan.cuh -- order-preserving block scans and a three-phase device-wide exclusive scan.
#pragma once
#include "common.cuh"

#define IBM_SCAN_NT 256           // threads per scan block
#define IBM_SCAN_IPT 8            // items per thread
#define IBM_SCAN_TILE (IBM_SCAN_NT * IBM_SCAN_IPT)

// Exclusive scan of one value per thread across a block of IBM_SCAN_NT threads (1-D block).
__device__ __forceinline__ long long block_exscan(long long v, long long& total) {
    __shared__ long long wsum[IBM_SCAN_NT / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        long long s = lane < IBM_SCAN_NT / 32 ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            long long y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < IBM_SCAN_NT / 32) wsum[lane] = s;
    }
    __syncthreads();
    long long base = w > 0 ? wsum[w - 1] : 0;
    total = wsum[IBM_SCAN_NT / 32 - 1];
    __syncthreads();
    return base + x - v;
}

// Phase 2: exclusive scan of the per-tile totals in place (one block of IBM_SCAN_NT threads),
// grand total in *total.
static __global__ void __launch_bounds__(IBM_SCAN_NT) k_scan_tile_totals(long long* __restrict__ t,
                                                                         long long ntiles, long long* total) {
    long long carry = 0;
    for (long long base = 0; base < ntiles; base += IBM_SCAN_TILE) {
        const long long b0 = base + (long long)threadIdx.x * IBM_SCAN_IPT;
        long long v[IBM_SCAN_IPT], s = 0;
#pragma unroll
        for (int q = 0; q < IBM_SCAN_IPT; ++q) {
            v[q] = b0 + q < ntiles ? t[b0 + q] : 0;
            s += v[q];
        }
        long long tot;
        long long off = carry + block_exscan(s, tot);
#pragma unroll
        for (int q = 0; q < IBM_SCAN_IPT; ++q) {
            if (b0 + q < ntiles) t[b0 + q] = off;
            off += v[q];
        }
        carry += tot;
    }
    if (threadIdx.x == 0) *total = carry;
}

// Count-then-write helpers: Count(i) gives the count of element i (i < n); tiles of IBM_SCAN_TILE
// consecutive elements are scanned independently and offset by the scanned tile totals.
template <class Count>
__global__ void __launch_bounds__(IBM_SCAN_NT) k_tile_totals(long long n, Count cnt, long long* __restrict__ tiles) {
    const long long base = (long long)blockIdx.x * IBM_SCAN_TILE + (long long)threadIdx.x * IBM_SCAN_IPT;
    long long s = 0;
#pragma unroll
    for (int q = 0; q < IBM_SCAN_IPT; ++q) {
        long long i = base + q;
        if (i < n) s += cnt(i);
    }
    long long tot;
    block_exscan(s, tot);
    if (threadIdx.x == 0) tiles[blockIdx.x] = tot;
}

// Calls emit(i, offset_i, count_i) for every element with its global exclusive offset.
template <class Count, class Emit>
__global__ void __launch_bounds__(IBM_SCAN_NT) k_tile_emit(long long n, Count cnt, Emit emit,
                                                          const long long* __restrict__ tiles) {
    const long long base = (long long)blockIdx.x * IBM_SCAN_TILE + (long long)threadIdx.x * IBM_SCAN_IPT;
    long long c[IBM_SCAN_IPT];
    long long s = 0;
#pragma unroll
    for (int q = 0; q < IBM_SCAN_IPT; ++q) {
        long long i = base + q;
        c[q] = i < n ? cnt(i) : 0;
        s += c[q];
    }
    long long tot;
    long long off = block_exscan(s, tot) + tiles[blockIdx.x];
#pragma unroll
    for (int q = 0; q < IBM_SCAN_IPT; ++q) {
        long long i = base + q;
        if (i < n) emit(i, off, c[q]);
        off += c[q];
    }
}

inline long long scan_tiles(long long n) { return (n + IBM_SCAN_TILE - 1) / IBM_SCAN_TILE; }

// Runs the three phases; tiles must hold scan_tiles(n) + 1 entries, d_total one entry.
template <class Count, class Emit>
inline cudaError_t scan_emit(long long n, Count cnt, Emit emit, long long* tiles, long long* d_total,
                             cudaStream_t s) {
    long long nt = scan_tiles(n);
    if (nt == 0) return cudaMemsetAsync(d_total, 0, sizeof(long long), s);
    k_tile_totals<<<(unsigned)nt, IBM_SCAN_NT, 0, s>>>(n, cnt, tiles);
    k_scan_tile_totals<<<1, IBM_SCAN_NT, 0, s>>>(tiles, nt, d_total);
    k_tile_emit<<<(unsigned)nt, IBM_SCAN_NT, 0, s>>>(n, cnt, emit, tiles);
    return cudaGetLastError();
}
