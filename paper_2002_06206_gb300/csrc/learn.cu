// learn.cu -- learned initial guess of the pressure Poisson solve: a small 3-D convolutional network
// (three 3x3x3 convolutions, 8 -> 8 -> 8 -> 1 channels, ReLU between) on the solver's grid that
// predicts how far p^{n+1} departs from the linear extrapolation 2 p^n - p^{n-1}, from the right-hand
// side, the last pressure change and the solid mask.  Activations and gradients are stored in BF16,
// channel-last (8 channels = 16 bytes per cell); the convolutions run as implicit GEMMs on the tensor
// cores (ldmatrix + mma.sync m16n8k16, BF16 operands, FP32 accumulation): M = 16 consecutive cells of
// a row, N = 8 channels, K = 27 taps x 8 channels (padded to 224).  The weight gradient is a reduction
// over all cells, done on the CUDA cores in FP32 with per-block partial sums reduced in a fixed order.
#include <cuda_bf16.h>
#include <math.h>

#include "solver.cuh"

#define NN_C 8
#define NN_TAPS 27
#define NN_KSTEPS 14            // 224 / 16
#define NN_NPARAM (2 * NN_C * NN_TAPS * NN_C + NN_TAPS * NN_C + 2 * NN_C + 1)

// Per-layer weights: W[co][tap][ci] (layer 3 has co = 1), bias[co].
struct NetParams {
    float* w[3];
    float* b[3];
};

struct ibm_net {
    float* master;            // NN_NPARAM FP32 parameters (W1, W2, W3, b1, b2, b3)
    float* grad;              // gradients, same layout
    float* m;                 // Adam moments
    float* v;
    uint32_t* frag_fwd[3];    // packed BF16 B fragments: [14 k-steps][32 lanes][2 regs]
    uint32_t* frag_bwd[3];    // fragments of the transposed weights (input-gradient convolution)
    long long step;
    // per-grid buffers (resized on demand by the host calls that receive a grid)
    long long cap_cells;
    __nv_bfloat16* x0;        // features
    __nv_bfloat16* y1;
    __nv_bfloat16* y2;
    __nv_bfloat16* d3;        // 2 (out - target) in channel 0
    __nv_bfloat16* d2;
    __nv_bfloat16* d1;
    float* out;
    float* wpart;             // per-block weight-gradient partials
    long long wpart_blocks;
    double* scal;             // [0] feature scale s, [1] loss sum, [2..] reduction scratch
    double* partials;
    unsigned* counter;
};

namespace {

__device__ __forceinline__ int tap_off(int t, int& dz, int& dy, int& dx) {
    dz = t / 9 - 1;
    dy = (t / 3) % 3 - 1;
    dx = t % 3 - 1;
    return 0;
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ void mma_bf16(float d[4], const uint32_t a[4], const uint32_t b[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Convolution of a channel-last BF16 field with 27 taps on the tensor cores (implicit GEMM, K = 27
// taps x 8 channels padded to 224).  sgn = +1: forward (input at c + off); sgn = -1: input gradient
// (input at c - off, transposed weights).  mode 0: store BF16 relu(acc + bias); mode 1: store FP32
// channel 0 of acc + bias; mode 2: store BF16 acc masked by (mask > 0) at the output cell (ReLU
// derivative).  The input is staged in shared memory.  A block owns a 32 x 4 (x, y) tile
// of output cells and walks NC_KZ planes; the input planes k - 1, k, k + 1 over the tile plus a one-cell
// halo sit in a three-plane ring (16 bytes per cell, zero outside the grid).  Warp w computes the
// 16 cells (w % 2) * 16 .. + 15 of row w / 2: for each k-step (two taps x 8 channels) one
// ldmatrix.x4 gathers the A fragment straight from the ring -- each lane names one 16-byte row, the
// input cell of its (cell, tap) -- and one mma.sync accumulates it.
#define NC_TX 32
#define NC_TY 4
#define NC_KZ 8
#define NC_SX (NC_TX + 2)
#define NC_SY (NC_TY + 2)
#define NC_PL (NC_SX * NC_SY)

__device__ __forceinline__ void ldsm_x4(uint32_t r[4], uint32_t addr) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
}

__global__ void __launch_bounds__(256) k_nn_conv_tile(int nx, int ny, int nz, const __nv_bfloat16* __restrict__ in,
                                                      const uint32_t* __restrict__ frag, const float* __restrict__ bias,
                                                      int sgn, int mode, __nv_bfloat16* __restrict__ outb,
                                                      float* __restrict__ outf, const __nv_bfloat16* __restrict__ mask) {
    __shared__ __align__(16) uint4 ring[3 * NC_PL + 1];          // + one zero row for the padding tap
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int x0 = blockIdx.x * NC_TX, y0 = blockIdx.y * NC_TY, z0 = blockIdx.z * NC_KZ;
    const int z1 = z0 + NC_KZ < nz ? z0 + NC_KZ : nz;
    if (tid == 0) ring[3 * NC_PL] = make_uint4(0u, 0u, 0u, 0u);
    auto load_plane = [&](int kk) {
        uint4* dst = ring + ((kk % 3) + 3) % 3 * NC_PL;
        for (int e = tid; e < NC_PL; e += 256) {
            const int gx = x0 + e % NC_SX - 1, gy = y0 + e / NC_SX - 1;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (kk >= 0 && kk < nz && gx >= 0 && gx < nx && gy >= 0 && gy < ny)
                v = *reinterpret_cast<const uint4*>(in + (gx + (long long)nx * (gy + (long long)ny * kk)) * NN_C);
            dst[e] = v;
        }
    };
    const int g = lane >> 2, q = lane & 3;
    uint32_t bf[NN_KSTEPS][2];
#pragma unroll
    for (int s = 0; s < NN_KSTEPS; ++s) {
        bf[s][0] = frag[(s * 32 + lane) * 2 + 0];
        bf[s][1] = frag[(s * 32 + lane) * 2 + 1];
    }
    const float b0 = bias ? bias[2 * q] : 0.f, b1 = bias ? bias[2 * q + 1] : 0.f;
    // this lane's ldmatrix row: matrix mj = lane / 8 (cells +8 for odd mj, tap +1 for mj >= 2), row lane % 8
    const int mj = lane >> 3, mr = lane & 7;
    const int cx = (w & 1) * 16 + ((mj & 1) ? 8 : 0) + mr;          // tile-local output x of the row
    const int cy = w >> 1;
    const uint32_t ring_base = (uint32_t)__cvta_generic_to_shared(ring);
    const uint32_t zero_row = ring_base + 3 * NC_PL * 16;
    load_plane(z0 - 1);
    load_plane(z0);
    for (int k = z0; k < z1; ++k) {
        load_plane(k + 1);
        __syncthreads();
        float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int s = 0; s < NN_KSTEPS; ++s) {
            const int t = 2 * s + (mj >> 1);
            uint32_t addr = zero_row;
            if (t < NN_TAPS) {
                int dz, dy, dx;
                tap_off(t, dz, dy, dx);
                const int sl = (((k + sgn * dz) % 3) + 3) % 3;
                addr = ring_base + (uint32_t)((sl * NC_PL + (cy + sgn * dy + 1) * NC_SX + (cx + sgn * dx + 1)) * 16);
            }
            uint32_t a[4];
            ldsm_x4(a, addr);
            // ldmatrix returns the matrices in lane order: 0 cells 0-7 tap 2s, 1 cells 8-15 tap 2s,
            // 2 cells 0-7 tap 2s+1, 3 cells 8-15 tap 2s+1 -- the a0..a3 order of mma's A fragment
            mma_bf16(d, a, bf[s]);
        }
        const int j = y0 + cy;
        const long long row = (long long)nx * (j + (long long)ny * k);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int i = x0 + (w & 1) * 16 + g + 8 * h;
            if (i >= nx || j >= ny) continue;
            const long long c = row + i;
            float v0 = d[2 * h] + b0, v1 = d[2 * h + 1] + b1;
            if (mode == 0) {
                v0 = fmaxf(v0, 0.f);
                v1 = fmaxf(v1, 0.f);
                *reinterpret_cast<uint32_t*>(outb + c * NN_C + 2 * q) = pack_bf16(v0, v1);
            } else if (mode == 1) {
                if (q == 0) outf[c] = v0;
            } else {
                const __nv_bfloat162 mk = *reinterpret_cast<const __nv_bfloat162*>(mask + c * NN_C + 2 * q);
                if (!(__bfloat162float(mk.x) > 0.f)) v0 = 0.f;
                if (!(__bfloat162float(mk.y) > 0.f)) v1 = 0.f;
                *reinterpret_cast<uint32_t*>(outb + c * NN_C + 2 * q) = pack_bf16(v0, v1);
            }
        }
        __syncthreads();
    }
}

// Weight and bias gradients of one layer: dW[co][tap][ci] = sum_c dz[c][co] y[c + off(tap)][ci],
// db[co] = sum_c dz[c][co].  Block = 224 threads: thread (tap, ci) for tid < 216, bias co for the
// last 8; each block covers a contiguous range of cells and writes its partial sums.
__global__ void __launch_bounds__(224) k_nn_wgrad(int nx, int ny, int nz, int ncout,
                                                  const __nv_bfloat16* __restrict__ dz,
                                                  const __nv_bfloat16* __restrict__ y, long long cells_per_block,
                                                  float* __restrict__ wpart) {
    const long long N = (long long)nx * ny * nz;
    const long long c0 = blockIdx.x * cells_per_block, c1 = c0 + cells_per_block < N ? c0 + cells_per_block : N;
    const int tid = threadIdx.x;
    float acc[NN_C] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const int t = tid / NN_C, ci = tid % NN_C;
    int dz_, dy_, dx_;
    tap_off(t < NN_TAPS ? t : 13, dz_, dy_, dx_);
    for (long long c = c0; c < c1; ++c) {
        const uint4 zv = *reinterpret_cast<const uint4*>(dz + c * NN_C);
        const __nv_bfloat162* zp = reinterpret_cast<const __nv_bfloat162*>(&zv);
        float zf[NN_C];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            zf[2 * h] = __bfloat162float(zp[h].x);
            zf[2 * h + 1] = __bfloat162float(zp[h].y);
        }
        float yv;
        if (tid < NN_TAPS * NN_C) {
            const int i = (int)(c % nx), j = (int)((c / nx) % ny), k = (int)(c / ((long long)nx * ny));
            const int ii = i + dx_, jj = j + dy_, kk = k + dz_;
            yv = (ii < 0 || ii >= nx || jj < 0 || jj >= ny || kk < 0 || kk >= nz)
                     ? 0.f
                     : __bfloat162float(y[(ii + (long long)nx * (jj + (long long)ny * kk)) * NN_C + ci]);
        } else {
            yv = 1.f;   // bias: sum of dz[co] with co = tid - 216
        }
#pragma unroll
        for (int co = 0; co < NN_C; ++co) acc[co] += zf[co] * yv;
    }
    float* part = wpart + (long long)blockIdx.x * (NN_TAPS * NN_C * NN_C + NN_C);
    if (tid < NN_TAPS * NN_C) {
        for (int co = 0; co < ncout; ++co) part[(co * NN_TAPS + t) * NN_C + ci] = acc[co];
    } else {
        const int co = tid - NN_TAPS * NN_C;
        part[NN_TAPS * NN_C * NN_C + co] = co < ncout ? acc[co] : 0.f;
    }
}

// Sums the per-block partials in block order; writes dW / db of the layer into grad (scaled by 1/N).
__global__ void k_nn_wgrad_reduce(const float* __restrict__ wpart, long long nblk, int ncout, float inv_n,
                                  float* __restrict__ gw, float* __restrict__ gb) {
    const int stride = NN_TAPS * NN_C * NN_C + NN_C;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < stride; e += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (long long b = 0; b < nblk; ++b) s += wpart[b * stride + e];
        if (e < NN_TAPS * NN_C * NN_C) {
            const int co = e / (NN_TAPS * NN_C);
            if (co < ncout) gw[e] = (float)(s * inv_n);
        } else {
            const int co = e - NN_TAPS * NN_C * NN_C;
            if (co < ncout) gb[co] = (float)(s * inv_n);
        }
    }
}

// Packs the BF16 B fragments of m16n8k16 for one layer.  Forward: B[kk][n] = W[n][tap][ci] with
// kk = 8 tap + ci.  Input gradient: B[kk][n] = W[co][tap][n] with kk = 8 tap + co.
__global__ void k_nn_pack(const float* __restrict__ w, int ncout, uint32_t* __restrict__ ffwd, uint32_t* __restrict__ fbwd) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;   // (kstep, lane)
    if (idx >= NN_KSTEPS * 32) return;
    const int s = idx / 32, lane = idx % 32, g = lane >> 2, q = lane & 3;
    for (int r = 0; r < 2; ++r) {
        const int kk0 = 16 * s + 8 * r + 2 * q;     // rows kk0, kk0 + 1
        float f[2], bw[2];
        for (int e = 0; e < 2; ++e) {
            const int kk = kk0 + e, t = kk / NN_C, c = kk % NN_C;
            f[e] = (t < NN_TAPS && g < ncout) ? w[(g * NN_TAPS + t) * NN_C + c] : 0.f;
            bw[e] = (t < NN_TAPS && c < ncout) ? w[(c * NN_TAPS + t) * NN_C + g] : 0.f;
        }
        ffwd[idx * 2 + r] = pack_bf16(f[0], f[1]);
        fbwd[idx * 2 + r] = pack_bf16(bw[0], bw[1]);
    }
}

// Features of a snapshot: channel 0 = b dx^2 / s, 1 = (p - p_prev) / s, 2 = 1 on cells with a cut link;
// s = RMS of p - p_prev (or of b dx^2 when the pressure has not moved), read from scal[0].
__global__ void k_nn_features(long long N, const double* __restrict__ b, const double* __restrict__ p,
                              const double* __restrict__ pp, const uint8_t* __restrict__ flags, double dx2,
                              const double* __restrict__ scal, __nv_bfloat16* __restrict__ x) {
    const double inv = scal[0] > 0.0 ? 1.0 / scal[0] : 0.0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        const float f0 = (float)(b[c] * dx2 * inv), f1 = (float)((p[c] - pp[c]) * inv);
        const float f2 = (flags && (flags[c] & 63u)) ? 1.f : 0.f;
        uint4 v;
        v.x = pack_bf16(f0, f1);
        v.y = pack_bf16(f2, 0.f);
        v.z = 0u;
        v.w = 0u;
        *reinterpret_cast<uint4*>(x + c * NN_C) = v;
    }
}

// scal[0] = RMS of (p - p_prev), or of b dx^2 if that is zero.
__global__ void k_nn_scale(long long N, const double* __restrict__ b, const double* __restrict__ p,
                           const double* __restrict__ pp, double dx2, double* partials, unsigned* counter,
                           double* scal) {
    float a0 = 0.f, a1 = 0.f;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        const float dp = (float)(p[c] - pp[c]);
        const float bb = (float)(b[c] * dx2);
        a0 += dp * dp;
        a1 += bb * bb;
    }
    double acc[2] = {(double)a0, (double)a1};
    grid_reduce<2>(acc, partials, counter, [&](double* t) {
        const double r0 = sqrt(t[0] / (double)N), r1 = sqrt(t[1] / (double)N);
        scal[0] = r0 > 0.0 ? r0 : (r1 > 0.0 ? r1 : 1.0);
    });
}

// Loss gradient seed: d3 channel 0 = 2 (out - target), others 0; the loss sum goes to scal[1].
__global__ void k_nn_loss(long long N, const float* __restrict__ out, const float* __restrict__ target,
                          __nv_bfloat16* __restrict__ d3, double* partials, unsigned* counter, double* scal) {
    float a = 0.f;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        const float e = out[c] - target[c];
        a += e * e;
        uint4 v;
        v.x = pack_bf16(2.f * e, 0.f);
        v.y = v.z = v.w = 0u;
        *reinterpret_cast<uint4*>(d3 + c * NN_C) = v;
    }
    double acc[1] = {(double)a};
    grid_reduce<1>(acc, partials, counter, [&](double* t) { scal[1] = t[0]; });
}

__global__ void k_nn_adam(int n, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                          float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const float gi = g[e];
        const float mi = b1 * m[e] + (1.f - b1) * gi;
        const float vi = b2 * v[e] + (1.f - b2) * gi * gi;
        m[e] = mi;
        v[e] = vi;
        p[e] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// x_guess = p + s * out
// Guess = linear extrapolation 2 p^n - p^{n-1} plus the network's scaled correction.
__global__ void k_nn_apply(long long N, const double* __restrict__ p, const double* __restrict__ pprev,
                           const float* __restrict__ out, const double* __restrict__ scal, double* __restrict__ xg) {
    const double s = scal[0];
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x)
        xg[c] = (2.0 * p[c] - pprev[c]) + s * (double)out[c];
}

unsigned blocks_n(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    long long cap = 8LL * IBM_NSM;
    if (b > cap) b = cap;
    return (unsigned)(b < 1 ? 1 : b);
}

long long offset_w(int l) { return l == 0 ? 0 : (l == 1 ? NN_C * NN_TAPS * NN_C : 2 * NN_C * NN_TAPS * NN_C); }
long long offset_b(int l) { return 2 * NN_C * NN_TAPS * NN_C + NN_TAPS * NN_C + l * NN_C; }
int cout_of(int l) { return l == 2 ? 1 : NN_C; }

// The training target of a snapshot, (p^{n+1} - 2 p^n + p^{n-1}) / s, formed in FP64 and stored in FP32.
__global__ void k_net_target(long long N, const double* __restrict__ pnext, const double* __restrict__ p,
                             const double* __restrict__ pprev, double s, float* __restrict__ out) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < N; q += (long long)gridDim.x * blockDim.x)
        out[q] = (float)((pnext[q] - 2.0 * p[q] + pprev[q]) / s);
}

}  // namespace

// ---- host side -----------------------------------------------------------------------------------

static int net_reserve(ibm_net* n, long long N) {
    if (N <= n->cap_cells) return IBM_OK;
    cudaFree(n->x0); cudaFree(n->y1); cudaFree(n->y2); cudaFree(n->d3); cudaFree(n->d2); cudaFree(n->d1);
    cudaFree(n->out); cudaFree(n->wpart);
    n->x0 = n->y1 = n->y2 = n->d3 = n->d2 = n->d1 = nullptr;
    n->out = n->wpart = nullptr;
    n->cap_cells = 0;
    const size_t act = (size_t)N * NN_C * sizeof(__nv_bfloat16);
    const long long nblk = (N + 4095) / 4096;
    cudaError_t e;
    if ((e = cudaMalloc(&n->x0, act)) != cudaSuccess || (e = cudaMalloc(&n->y1, act)) != cudaSuccess ||
        (e = cudaMalloc(&n->y2, act)) != cudaSuccess || (e = cudaMalloc(&n->d3, act)) != cudaSuccess ||
        (e = cudaMalloc(&n->d2, act)) != cudaSuccess || (e = cudaMalloc(&n->d1, act)) != cudaSuccess ||
        (e = cudaMalloc(&n->out, (size_t)N * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&n->wpart, (size_t)nblk * (NN_TAPS * NN_C * NN_C + NN_C) * sizeof(float))) != cudaSuccess)
        return ibm_fail(IBM_E_NOMEM, "ibm_net: %s", cudaGetErrorString(e));
    n->cap_cells = N;
    n->wpart_blocks = nblk;
    return IBM_OK;
}

extern "C" void ibm_net_destroy(ibm_net* n) {
    if (!n) return;
    cudaFree(n->master); cudaFree(n->grad); cudaFree(n->m); cudaFree(n->v);
    for (int l = 0; l < 3; ++l) { cudaFree(n->frag_fwd[l]); cudaFree(n->frag_bwd[l]); }
    cudaFree(n->x0); cudaFree(n->y1); cudaFree(n->y2); cudaFree(n->d3); cudaFree(n->d2); cudaFree(n->d1);
    cudaFree(n->out); cudaFree(n->wpart); cudaFree(n->scal); cudaFree(n->partials); cudaFree(n->counter);
    free(n);
}

static int net_pack(ibm_net* n, cudaStream_t s) {
    for (int l = 0; l < 3; ++l)
        k_nn_pack<<<(NN_KSTEPS * 32 + 127) / 128, 128, 0, s>>>(n->master + offset_w(l), cout_of(l), n->frag_fwd[l],
                                                                n->frag_bwd[l]);
    IBM_LAUNCHED("ibm_net: pack");
    return IBM_OK;
}

extern "C" int ibm_net_create(const float* h_params, ibm_net** out) {
    if (!out) return ibm_fail(IBM_E_INVALID, "ibm_net_create: null output");
    *out = nullptr;
    ibm_net* n = (ibm_net*)calloc(1, sizeof(ibm_net));
    if (!n) return ibm_fail(IBM_E_NOMEM, "ibm_net_create: host allocation");
    cudaError_t e;
    const size_t pb = (NN_NPARAM + 16) * sizeof(float);   // padded: layer 3's bias is read as 8 lanes
    const size_t fb = NN_KSTEPS * 32 * 2 * sizeof(uint32_t);
    if ((e = cudaMalloc(&n->master, pb)) != cudaSuccess || (e = cudaMalloc(&n->grad, pb)) != cudaSuccess ||
        (e = cudaMalloc(&n->m, pb)) != cudaSuccess || (e = cudaMalloc(&n->v, pb)) != cudaSuccess ||
        (e = cudaMalloc(&n->scal, 8 * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&n->partials, 8 * 8 * IBM_NSM * sizeof(double) * 2)) != cudaSuccess ||
        (e = cudaMalloc(&n->counter, 4 * sizeof(unsigned))) != cudaSuccess) {
        ibm_net_destroy(n);
        return ibm_fail(IBM_E_NOMEM, "ibm_net_create: %s", cudaGetErrorString(e));
    }
    for (int l = 0; l < 3; ++l)
        if ((e = cudaMalloc(&n->frag_fwd[l], fb)) != cudaSuccess || (e = cudaMalloc(&n->frag_bwd[l], fb)) != cudaSuccess) {
            ibm_net_destroy(n);
            return ibm_fail(IBM_E_NOMEM, "ibm_net_create: %s", cudaGetErrorString(e));
        }
    if ((e = cudaMemset(n->m, 0, pb)) != cudaSuccess || (e = cudaMemset(n->v, 0, pb)) != cudaSuccess ||
        (e = cudaMemset(n->grad, 0, pb)) != cudaSuccess ||
        (e = cudaMemset(n->counter, 0, 4 * sizeof(unsigned))) != cudaSuccess ||
        (e = cudaMemset(n->scal, 0, 8 * sizeof(double))) != cudaSuccess ||
        (e = cudaMemset(n->master, 0, pb)) != cudaSuccess) {
        ibm_net_destroy(n);
        return ibm_cuda_check(e, "ibm_net_create");
    }
    if (h_params && (e = cudaMemcpy(n->master, h_params, NN_NPARAM * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess) {
        ibm_net_destroy(n);
        return ibm_cuda_check(e, "ibm_net_create");
    }
    int rc = net_pack(n, 0);
    if (!rc && (e = cudaDeviceSynchronize()) != cudaSuccess) rc = ibm_cuda_check(e, "ibm_net_create");
    if (rc) {
        ibm_net_destroy(n);
        return rc;
    }
    *out = n;
    return IBM_OK;
}

extern "C" int ibm_net_num_params(void) { return NN_NPARAM; }

extern "C" int ibm_net_get_params(const ibm_net* n, float* h_params) {
    if (!n || !h_params) return ibm_fail(IBM_E_INVALID, "ibm_net_get_params: null argument");
    IBM_CUDA(cudaMemcpy(h_params, n->master, NN_NPARAM * sizeof(float), cudaMemcpyDeviceToHost));
    return IBM_OK;
}

extern "C" int ibm_net_get_grads(const ibm_net* n, float* h_grads) {
    if (!n || !h_grads) return ibm_fail(IBM_E_INVALID, "ibm_net_get_grads: null argument");
    IBM_CUDA(cudaMemcpy(h_grads, n->grad, NN_NPARAM * sizeof(float), cudaMemcpyDeviceToHost));
    return IBM_OK;
}

static void conv(const ibm_net* n, int nx, int ny, int nz, const __nv_bfloat16* in, int l, int sgn, int mode,
                 __nv_bfloat16* outb, float* outf, const __nv_bfloat16* mask, cudaStream_t s) {
    const dim3 grid((unsigned)((nx + NC_TX - 1) / NC_TX), (unsigned)((ny + NC_TY - 1) / NC_TY),
                    (unsigned)((nz + NC_KZ - 1) / NC_KZ));
    k_nn_conv_tile<<<grid, 256, 0, s>>>(nx, ny, nz, in, sgn > 0 ? n->frag_fwd[l] : n->frag_bwd[l],
                                        sgn > 0 ? n->master + offset_b(l) : nullptr, sgn, mode, outb, outf, mask);
}

static int net_forward(ibm_net* n, const ibm_grid* g, cudaStream_t s) {
    conv(n, g->nx, g->ny, g->nz, n->x0, 0, +1, 0, n->y1, nullptr, nullptr, s);
    conv(n, g->nx, g->ny, g->nz, n->y1, 1, +1, 0, n->y2, nullptr, nullptr, s);
    conv(n, g->nx, g->ny, g->nz, n->y2, 2, +1, 1, nullptr, n->out, nullptr, s);
    IBM_LAUNCHED("ibm_net: forward");
    return IBM_OK;
}

static int net_features(ibm_net* n, const ibm_grid* g, const double* b, const double* p, const double* pprev,
                        const uint8_t* flags, cudaStream_t s) {
    const long long N = (long long)g->nx * g->ny * g->nz;
    int rc = net_reserve(n, N);
    if (rc) return rc;
    const double dx2 = g->dx * g->dx;
    k_nn_scale<<<blocks_n(N, 256), 256, 0, s>>>(N, b, p, pprev, dx2, n->partials, n->counter, n->scal);
    k_nn_features<<<blocks_n(N, 256), 256, 0, s>>>(N, b, p, pprev, flags, dx2, n->scal, n->x0);
    IBM_LAUNCHED("ibm_net: features");
    return IBM_OK;
}

// Forward pass on a snapshot: d_out[N] (float) = the network's normalised pressure change; *scale
// (host, may be NULL, synchronises) = the normalisation s.
extern "C" int ibm_net_forward(ibm_net* n, const ibm_grid* g, const double* d_b, const double* d_p,
                               const double* d_pprev, const uint8_t* d_flags, float* d_out, double* scale,
                               void* stream) {
    int rc = ibm_check_grid(g);
    if (rc) return rc;
    if (!n || !d_b || !d_p || !d_pprev) return ibm_fail(IBM_E_INVALID, "ibm_net_forward: null argument");
    cudaStream_t s = (cudaStream_t)stream;
    if ((rc = net_features(n, g, d_b, d_p, d_pprev, d_flags, s))) return rc;
    if ((rc = net_forward(n, g, s))) return rc;
    const long long N = (long long)g->nx * g->ny * g->nz;
    if (d_out) IBM_CUDA(cudaMemcpyAsync(d_out, n->out, N * sizeof(float), cudaMemcpyDeviceToDevice, s));
    if (scale) {
        IBM_CUDA(cudaMemcpyAsync(scale, n->scal, sizeof(double), cudaMemcpyDeviceToHost, s));
        IBM_CUDA(cudaStreamSynchronize(s));
    }
    return IBM_OK;
}

// The training target of a snapshot: d_target[N] = (p_next - 2 p + p_prev) / s in FP32, s the scale that
// ibm_net_forward returned for (b, p, p_prev).
extern "C" int ibm_net_target(const ibm_grid* g, const double* d_pnext, const double* d_p, const double* d_pprev,
                              double s, float* d_target, void* stream) {
    int rc = ibm_check_grid(g);
    if (rc) return rc;
    if (!d_pnext || !d_p || !d_pprev || !d_target) return ibm_fail(IBM_E_INVALID, "ibm_net_target: null argument");
    if (!(s > 0.0) || !isfinite(s)) return ibm_fail(IBM_E_INVALID, "ibm_net_target: the scale must be positive");
    const long long N = (long long)g->nx * g->ny * g->nz;
    k_net_target<<<blocks_n(N, 256), 256, 0, (cudaStream_t)stream>>>(N, d_pnext, d_p, d_pprev, s, d_target);
    IBM_LAUNCHED("ibm_net: target");
    IBM_CUDA(cudaGetLastError());
    return IBM_OK;
}

// One training step on a snapshot: features from (b, p, p_prev, flags) against the target of
// ibm_net_target, forward, mean squared error, backward, Adam (lr; betas 0.9, 0.999).  *loss (host,
// synchronises) = the mean squared error before the update.  lr = 0 computes the gradients only.
extern "C" int ibm_net_train_step(ibm_net* n, const ibm_grid* g, const double* d_b, const double* d_p,
                                  const double* d_pprev, const uint8_t* d_flags, const float* d_target, float lr,
                                  double* loss, void* stream) {
    int rc = ibm_check_grid(g);
    if (rc) return rc;
    if (!n || !d_b || !d_p || !d_pprev || !d_target) return ibm_fail(IBM_E_INVALID, "ibm_net_train_step: null argument");
    cudaStream_t s = (cudaStream_t)stream;
    const long long N = (long long)g->nx * g->ny * g->nz;
    if ((rc = net_features(n, g, d_b, d_p, d_pprev, d_flags, s))) return rc;
    if ((rc = net_forward(n, g, s))) return rc;
    k_nn_loss<<<blocks_n(N, 256), 256, 0, s>>>(N, n->out, d_target, n->d3, n->partials, n->counter, n->scal);
    // input gradients (ReLU derivative of the layer below applied at the output cell)
    conv(n, g->nx, g->ny, g->nz, n->d3, 2, -1, 2, n->d2, nullptr, n->y2, s);
    conv(n, g->nx, g->ny, g->nz, n->d2, 1, -1, 2, n->d1, nullptr, n->y1, s);
    // weight gradients
    const long long cpb = 4096;
    const unsigned nblk = (unsigned)((N + cpb - 1) / cpb);
    const __nv_bfloat16* dz[3] = {n->d1, n->d2, n->d3};
    const __nv_bfloat16* yin[3] = {n->x0, n->y1, n->y2};
    for (int l = 0; l < 3; ++l) {
        k_nn_wgrad<<<nblk, 224, 0, s>>>(g->nx, g->ny, g->nz, cout_of(l), dz[l], yin[l], cpb, n->wpart);
        k_nn_wgrad_reduce<<<8, 256, 0, s>>>(n->wpart, nblk, cout_of(l), 1.f / (float)N, n->grad + offset_w(l),
                                            n->grad + offset_b(l));
    }
    IBM_LAUNCHED("ibm_net: backward");
    if (lr > 0.f) {
        n->step += 1;
        const float c1 = 1.f - powf(0.9f, (float)n->step), c2 = 1.f - powf(0.999f, (float)n->step);
        k_nn_adam<<<(NN_NPARAM + 255) / 256, 256, 0, s>>>(NN_NPARAM, n->master, n->grad, n->m, n->v, lr, 0.9f, 0.999f,
                                                          1e-8f, c1, c2);
        if ((rc = net_pack(n, s))) return rc;
    }
    if (loss) {
        double h[2];
        IBM_CUDA(cudaMemcpyAsync(h, n->scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
        IBM_CUDA(cudaStreamSynchronize(s));
        *loss = h[1] / (double)N;
    }
    return IBM_OK;
}

// x_guess = p + s * net(b, p, p_prev, flags) on the state's grid (used by les_step).
int net_guess(ibm_net* n, const ibm_grid* g, const double* b, const double* p, const double* pprev,
              const uint8_t* flags, double* xg, cudaStream_t s) {
    int rc = net_features(n, g, b, p, pprev, flags, s);
    if (rc) return rc;
    if ((rc = net_forward(n, g, s))) return rc;
    const long long N = (long long)g->nx * g->ny * g->nz;
    k_nn_apply<<<blocks_n(N, 256), 256, 0, s>>>(N, p, pprev, n->out, n->scal, xg);
    IBM_LAUNCHED("ibm_net: guess");
    return IBM_OK;
}
