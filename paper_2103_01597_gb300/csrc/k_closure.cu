// Learned closure for a 2x-coarser grid: restriction of a fine state, and a
// three-layer 3-D conv net (8 -> 32 -> 32 -> 8 channels, 3x3x3 kernels,
// circular padding, ReLU between layers) with its forward pass, hand-written
// backward pass, Adam update and the guarded application of its correction to
// a coarse state.  The paper only mentions machine-learned reconstruction of
// turbulent flows from low-resolution data (Sec. 6); everything here is a
// reading of that remark.
//
// Convolutions are implicit GEMMs on the tensor cores with bfloat16 operands
// and binary32 accumulation (mma.sync m16n8k16): M = 128 cells of an x-row,
// N = output channels, K = 27 taps x input channels.  The row tile with a
// one-cell halo is staged once per (dy, dz) tap group and serves the three dx
// taps by shifting the window.  Activations are channel-major [C][N]
// (N = nx ny nz, x fastest), like the solver's fields.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <new>

#include "ac_internal.h"
#include "conv_tc.cuh"
#include "wgrad_tc.cuh"

namespace ac {

using bf16 = __nv_bfloat16;

constexpr int CL_TM = 128;       // cells per CTA tile
constexpr int CL_THREADS = 128;  // four warps, 32 cells each
constexpr int CL_WG_CTAS = 64;   // CTAs per tap group in the weight-gradient kernel

struct ConvGeom {
    int nx, ny, nz;
    long long n;  // cells
};

__device__ __forceinline__ int cl_wrap(int v, int n) {
    int m = v % n;
    return m < 0 ? m + n : m;
}

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const unsigned (&a)[4],
                                               const unsigned (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ unsigned pack_bf16(bf16 lo, bf16 hi) {
    return (unsigned)__bfloat16_as_ushort(lo) | ((unsigned)__bfloat16_as_ushort(hi) << 16);
}

enum { EPI_RELU_BF16 = 0, EPI_LINEAR_F32 = 1, EPI_MASK_BF16 = 2 };

// y[co, p] = sum_{tap, ci} Wt[co][tap][ci] x[ci, p + off(tap)]  (+ epilogue):
//   EPI_RELU_BF16:  max(y + bias, 0) as bfloat16 (hidden layers);
//   EPI_LINEAR_F32: y + bias as binary32 (output layer);
//   EPI_MASK_BF16:  y where mask > 0, else 0, as bfloat16 (input gradient
//                   through a ReLU, with flipped/transposed weights).
template <int CIN, int COUT, int EPI>
__global__ void __launch_bounds__(CL_THREADS) conv_fwd_kernel(const bf16 *__restrict__ X,
                                                              const bf16 *__restrict__ Wt,
                                                              const float *__restrict__ bias,
                                                              const bf16 *__restrict__ mask,
                                                              void *__restrict__ Y, ConvGeom g) {
    constexpr int PA = CIN + 8;  // padded pitches keep the fragment loads conflict-free
    constexpr int KG = 3 * CIN;
    constexpr int PB = KG + 8;
    constexpr int NT = COUT / 8;
    __shared__ __align__(16) bf16 As[(CL_TM + 2) * PA];
    __shared__ __align__(16) bf16 Bs[COUT * PB];
    const int segs = (g.nx + CL_TM - 1) / CL_TM;
    const int row = blockIdx.x / segs;
    const int seg = blockIdx.x - row * segs;
    const int y = row % g.ny, z = row / g.ny;
    const int x0 = seg * CL_TM;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int gq = lane >> 2, tq = lane & 3;
    float acc[2][NT][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[mt][nt][r] = 0.f;

    for (int grp = 0; grp < 9; ++grp) {
        const int dz = grp / 3 - 1, dy = grp % 3 - 1;
        const long long rbase = ((long long)cl_wrap(z + dz, g.nz) * g.ny + cl_wrap(y + dy, g.ny)) * g.nx;
        __syncthreads();  // previous group's tiles are no longer read
        for (int idx = tid; idx < CIN * (CL_TM + 2); idx += CL_THREADS) {
            const int ci = idx / (CL_TM + 2);
            const int c = idx - ci * (CL_TM + 2);
            As[c * PA + ci] = X[(long long)ci * g.n + rbase + cl_wrap(x0 - 1 + c, g.nx)];
        }
        for (int idx = tid; idx < COUT * KG; idx += CL_THREADS) {
            const int co = idx / KG;
            const int r = idx - co * KG;
            const int j = r / CIN, ci = r - j * CIN;
            Bs[co * PB + r] = Wt[((long long)co * 27 + grp * 3 + j) * CIN + ci];
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < 3; ++j) {  // dx = j - 1: the window starts j cells into the halo tile
#pragma unroll
            for (int kk = 0; kk < CIN / 16; ++kk) {
                unsigned a[2][4];
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    const int r0 = warp * 32 + mt * 16 + gq + j;
                    const bf16 *p0 = As + r0 * PA + kk * 16 + 2 * tq;
                    const bf16 *p1 = p0 + 8 * PA;
                    a[mt][0] = *reinterpret_cast<const unsigned *>(p0);
                    a[mt][1] = *reinterpret_cast<const unsigned *>(p1);
                    a[mt][2] = *reinterpret_cast<const unsigned *>(p0 + 8);
                    a[mt][3] = *reinterpret_cast<const unsigned *>(p1 + 8);
                }
#pragma unroll
                for (int nt = 0; nt < NT; ++nt) {
                    const bf16 *pb = Bs + (nt * 8 + gq) * PB + j * CIN + kk * 16 + 2 * tq;
                    const unsigned b[2] = {*reinterpret_cast<const unsigned *>(pb),
                                           *reinterpret_cast<const unsigned *>(pb + 8)};
                    mma_bf16_16816(acc[0][nt], a[0], b);
                    mma_bf16_16816(acc[1][nt], a[1], b);
                }
            }
        }
    }
    const long long obase = ((long long)z * g.ny + y) * g.nx;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const int x = x0 + warp * 32 + mt * 16 + gq + 8 * h;
                    if (x >= g.nx) continue;
                    const int co = nt * 8 + 2 * tq + c;
                    const long long o = (long long)co * g.n + obase + x;
                    float v = acc[mt][nt][2 * h + c];
                    if (EPI == EPI_RELU_BF16) {
                        v = fmaxf(v + bias[co], 0.f);
                        static_cast<bf16 *>(Y)[o] = __float2bfloat16_rn(v);
                    } else if (EPI == EPI_LINEAR_F32) {
                        static_cast<float *>(Y)[o] = v + bias[co];
                    } else {
                        v = __bfloat162float(mask[o]) > 0.f ? v : 0.f;
                        static_cast<bf16 *>(Y)[o] = __float2bfloat16_rn(v);
                    }
                }
}

// Partial weight gradients of one tap group (blockIdx.y = dz, dy):
// part[grp][cta][co][j * CIN + ci] = sum over this CTA's cells of
// dZ[co, p] x[ci, p + off(dz, dy, j - 1)].  M = output channels (padded to 16),
// N = 3 CIN, K = cells.
template <int CIN, int COUT>
__global__ void __launch_bounds__(CL_THREADS) conv_wgrad_kernel(const bf16 *__restrict__ dZ,
                                                                const bf16 *__restrict__ X,
                                                                float *__restrict__ part,
                                                                ConvGeom g) {
    constexpr int MT = (COUT + 15) / 16;
    constexpr int KN = 3 * CIN;
    constexpr int NT = KN / 8;
    constexpr int NTW = (NT + 3) / 4;
    constexpr int PD = CL_TM + 8;
    constexpr int PX = CL_TM + 8;
    __shared__ __align__(16) bf16 Ds[MT * 16 * PD];
    __shared__ __align__(16) bf16 Xs[CIN * PX];
    const int grp = blockIdx.y;
    const int dz = grp / 3 - 1, dy = grp % 3 - 1;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int gq = lane >> 2, tq = lane & 3;
    float acc[MT][NTW][4];
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
        for (int w = 0; w < NTW; ++w)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[mt][w][r] = 0.f;
    const int segs = (g.nx + CL_TM - 1) / CL_TM;
    const long long tiles = (long long)g.ny * g.nz * segs;
    for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int row = (int)(tile / segs);
        const int seg = (int)(tile - (long long)row * segs);
        const int y = row % g.ny, z = row / g.ny;
        const int x0 = seg * CL_TM;
        const long long obase = ((long long)z * g.ny + y) * g.nx;
        const long long rbase = ((long long)cl_wrap(z + dz, g.nz) * g.ny + cl_wrap(y + dy, g.ny)) * g.nx;
        __syncthreads();
        for (int idx = tid; idx < MT * 16 * CL_TM; idx += CL_THREADS) {
            const int co = idx / CL_TM;
            const int c = idx - co * CL_TM;
            const int x = x0 + c;
            Ds[co * PD + c] = (co < COUT && x < g.nx) ? dZ[(long long)co * g.n + obase + x]
                                                      : __float2bfloat16_rn(0.f);
        }
        for (int idx = tid; idx < CIN * (CL_TM + 2); idx += CL_THREADS) {
            const int ci = idx / (CL_TM + 2);
            const int c = idx - ci * (CL_TM + 2);
            Xs[ci * PX + c] = X[(long long)ci * g.n + rbase + cl_wrap(x0 - 1 + c, g.nx)];
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < CL_TM / 16; ++ks) {
            unsigned a[MT][4];
#pragma unroll
            for (int mt = 0; mt < MT; ++mt) {
                const bf16 *p0 = Ds + (mt * 16 + gq) * PD + ks * 16 + 2 * tq;
                const bf16 *p1 = p0 + 8 * PD;
                a[mt][0] = *reinterpret_cast<const unsigned *>(p0);
                a[mt][1] = *reinterpret_cast<const unsigned *>(p1);
                a[mt][2] = *reinterpret_cast<const unsigned *>(p0 + 8);
                a[mt][3] = *reinterpret_cast<const unsigned *>(p1 + 8);
            }
#pragma unroll
            for (int w = 0; w < NTW; ++w) {
                const int nt = warp + 4 * w;
                if (nt >= NT) continue;
                const int nn = nt * 8 + gq;
                const int j = nn / CIN, ci = nn - (nn / CIN) * CIN;
                const bf16 *px = Xs + ci * PX + ks * 16 + 2 * tq + j;
                const unsigned b[2] = {pack_bf16(px[0], px[1]), pack_bf16(px[8], px[9])};
#pragma unroll
                for (int mt = 0; mt < MT; ++mt) mma_bf16_16816(acc[mt][w], a[mt], b);
            }
        }
    }
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
        for (int w = 0; w < NTW; ++w) {
            const int nt = warp + 4 * w;
            if (nt >= NT) continue;
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const int co = mt * 16 + gq + 8 * h;
                    if (co >= COUT) continue;
                    const int nn = nt * 8 + 2 * tq + c;
                    part[(((long long)grp * gridDim.x + blockIdx.x) * COUT + co) * KN + nn] =
                        acc[mt][w][2 * h + c];
                }
        }
}

// Sum the per-CTA partials into the gradient of W[co][ci][kz][ky][kx] (only the
// first cin_real input channels exist).
__global__ void wgrad_reduce_kernel(const float *__restrict__ part, int ctas, int cout, int cin,
                                    int cin_real, float *__restrict__ gW) {
    const int total = cout * cin_real * 27;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const int co = t / (cin_real * 27);
        const int rem = t - co * cin_real * 27;
        const int ci = rem / 27;
        const int tap = rem - ci * 27;
        const int grp = tap / 3, j = tap - grp * 3;
        double s = 0.0;
        for (int b = 0; b < ctas; ++b)
            s += part[(((long long)grp * ctas + b) * cout + co) * (3 * cin) + j * cin + ci];
        gW[t] = (float)s;
    }
}

// db[co] = sum over cells of dZ[co, p] (one block per channel, fixed order).
__global__ void bias_grad_kernel(const bf16 *__restrict__ dZ, long long n, float *__restrict__ gb) {
    const int co = blockIdx.x;
    double s = 0.0;
    for (long long p = threadIdx.x; p < n; p += blockDim.x)
        s += (double)__bfloat162float(dZ[(long long)co * n + p]);
    __shared__ double sh[256];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) gb[co] = (float)sh[0];
}

// Network input: x[c] = f[c] / in_scale[c] as bfloat16 (channels 8..15 stay zero).
struct F8 {
    const float *p[8];
};
struct W8 {
    float *p[8];
};
__global__ void pack_input_kernel(F8 f, const float *__restrict__ inv_scale, long long n,
                                  bf16 *__restrict__ x) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < 16 * n;
         t += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(t / n);
        const long long p = t - c * n;
        // channels 8..15 are zero padding (the buffer is shared with the row-planar layout)
        x[t] = c < 8 ? __float2bfloat16_rn(f.p[c][p] * inv_scale[c]) : __float2bfloat16_rn(0.f);
    }
}

// Loss and output gradient: d = y - target / out_scale; loss partial sums of
// d^2 (binary64); dY = 2 d / (8 n) as bfloat16.
__global__ void loss_grad_kernel(const float *__restrict__ y, F8 tgt,
                                 const float *__restrict__ inv_out, long long n,
                                 bf16 *__restrict__ dy, double *__restrict__ partials) {
    double acc = 0.0;
    const float gsc = (float)(2.0 / (8.0 * (double)n));
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < 8 * n;
         t += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(t / n);
        const long long p = t - c * n;
        const float d = y[t] - tgt.p[c][p] * inv_out[c];
        acc += (double)d * (double)d;
        dy[t] = __float2bfloat16_rn(gsc * d);
    }
    __shared__ double sh[256];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = sh[0];
}

// out[c] = out_scale[c] * y[c] (y channel-major [8][n])
__global__ void scale_output_kernel(const float *__restrict__ y, const float *__restrict__ out_scale,
                                    long long n, W8 out) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < 8 * n;
         t += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(t / n);
        out.p[c][t - c * n] = out_scale[c] * y[t];
    }
}

// Row-planar network input for the tensor-memory kernels (layout in conv_tc.cuh,
// one plane of 8 channels): f[c] / in_scale[c] as bfloat16; cells x = 0 and
// nx - 1 are also written to the periodic halo slots.
__global__ void pack_input_rp_kernel(F8 f, const float *__restrict__ inv_scale, int nx,
                                     long long n, bf16 *__restrict__ x) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        const long long row = p / nx;  // z * ny + y
        const int xi = (int)(p - row * nx);
        __align__(16) bf16 v[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) v[c] = __float2bfloat16_rn(f.p[c][p] * inv_scale[c]);
        const uint4 val = *reinterpret_cast<const uint4 *>(v);
        uint4 *p0 = reinterpret_cast<uint4 *>(x + row * tc::rp_cells(nx) * 8);
        p0[xi + 1] = val;
        if (xi == 0) p0[nx + 1] = val;
        if (xi == nx - 1) p0[0] = val;
    }
}

// Guard: largest |out_scale * y| (NaN counts as larger than anything) into one word.
__global__ void correction_max_kernel(const float *__restrict__ y,
                                      const float *__restrict__ out_scale, long long n,
                                      unsigned long long *gmax) {
    double m = 0.0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < 8 * n;
         t += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(t / n);
        const double v = fabs((double)(out_scale[c] * y[t]));
        m = (v > m || v != v) ? v : m;
    }
    unsigned long long bits = (unsigned long long)__double_as_longlong(m);
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long other = __shfl_xor_sync(0xffffffffu, bits, o);
        bits = other > bits ? other : bits;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(gmax, bits);
}

// f[c] += s[c] * y[c] (s = out_scale, or 1 where y is already scaled: s == null),
// only if the guard word shows a finite maximum <= limit.
__global__ void apply_correction_kernel(W8 f, const float *__restrict__ y,
                                        const float *__restrict__ out_scale, long long n,
                                        const unsigned long long *gmax, double limit) {
    const double m = __longlong_as_double((long long)*gmax);
    if (!(m <= limit)) return;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < 8 * n;
         t += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(t / n);
        f.p[c][t - c * n] += (out_scale ? out_scale[c] : 1.f) * y[t];
    }
}

// Adam (Kingma and Ba 2015) on the binary32 master parameters.
__global__ void adam_kernel(float *__restrict__ p, float *__restrict__ m, float *__restrict__ v,
                            const float *__restrict__ g, int n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const float gt = g[t];
        const float mt = b1 * m[t] + (1.f - b1) * gt;
        const float vt = b2 * v[t] + (1.f - b2) * gt * gt;
        m[t] = mt;
        v[t] = vt;
        p[t] -= lr * (mt / c1) / (sqrtf(vt / c2) + eps);
    }
}

// bfloat16 weights from the master copy W[co][ci][tap]:
//   forward layout    Wf[co][tap][ci_pad]   (ci >= cin stays zero);
//   transposed layout Wb[ci][26 - tap][co_pad] for the input gradient.
__global__ void prep_weights_kernel(const float *__restrict__ W, int cout, int cin, int cin_pad,
                                    bf16 *__restrict__ wf, int cout_pad, bf16 *__restrict__ wb) {
    const int total = cout * cin * 27;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const int co = t / (cin * 27);
        const int rem = t - co * cin * 27;
        const int ci = rem / 27;
        const int tap = rem - ci * 27;
        const bf16 w = __float2bfloat16_rn(W[t]);
        wf[((long long)co * 27 + tap) * cin_pad + ci] = w;
        if (wb) wb[((long long)ci * 27 + (26 - tap)) * cout_pad + co] = w;
    }
}

// Full-weighting restriction: coarse(I) = sum_d w(d) fine(2I + d), w = (1/4, 1/2, 1/4)
// per axis, periodic; binary64 accumulation, binary32 result.
template <typename T>
__global__ void restrict_kernel(const T *__restrict__ fine, int nxf, int nyf, int nzf,
                                float *__restrict__ coarse) {
    const int nxc = nxf / 2, nyc = nyf / 2, nzc = nzf / 2;
    const long long total = (long long)nxc * nyc * nzc;
    const double w[3] = {0.25, 0.5, 0.25};
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int I = (int)(t % nxc);
        const int J = (int)((t / nxc) % nyc);
        const int K = (int)(t / ((long long)nxc * nyc));
        double acc = 0.0;
        for (int dk = -1; dk <= 1; ++dk)
            for (int dj = -1; dj <= 1; ++dj)
                for (int di = -1; di <= 1; ++di) {
                    const long long idx =
                        ((long long)cl_wrap(2 * K + dk, nzf) * nyf + cl_wrap(2 * J + dj, nyf)) * nxf +
                        cl_wrap(2 * I + di, nxf);
                    acc += w[di + 1] * w[dj + 1] * w[dk + 1] * (double)fine[idx];
                }
        coarse[t] = (float)acc;
    }
}

// Loss and output gradient for the tcgen05 backward pass: as loss_grad_kernel,
// with dY (8 channels) written row-planar, with its periodic halo cells, twice:
// one plane (dyh, the input of the next convolution) and two planes (dy2h, the
// second zero: the weight-gradient operand, N padded to 16).  A cell's
// eight squares are summed in binary32, the cells' sums in binary64 (binary64
// work is slow on this part: one conversion and one add per cell); block
// partials of the loss in partials[blockIdx.x].
__global__ void loss_grad_rp_kernel(const float *__restrict__ y, F8 tgt,
                                    const float *__restrict__ inv_out, int nx, long long n,
                                    bf16 *__restrict__ dyh, bf16 *__restrict__ dy2h,
                                    double *__restrict__ partials) {
    double acc = 0.0;
    const float gsc = (float)(2.0 / (8.0 * (double)n));
    const long long nxp = tc::rp_cells(nx);
    const bool narrow = n <= 0xffffffffLL;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        const long long row = narrow ? (long long)((unsigned)p / (unsigned)nx) : p / nx;  // z * ny + y
        const int xi = (int)(p - row * nx);
        __align__(16) bf16 v[8];
        float sq = 0.f;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const float d = y[c * n + p] - tgt.p[c][p] * inv_out[c];
            sq = fmaf(d, d, sq);
            v[c] = __float2bfloat16_rn(gsc * d);
        }
        acc += (double)sq;
        const uint4 val = *reinterpret_cast<const uint4 *>(v);
        uint4 *h = reinterpret_cast<uint4 *>(dyh + row * nxp * 8);
        h[xi + 1] = val;
        if (xi == 0) h[nx + 1] = val;
        if (xi == nx - 1) h[0] = val;
        uint4 *h2 = reinterpret_cast<uint4 *>(dy2h + row * 2 * nxp * 8);
        h2[xi + 1] = val;
        if (xi == 0) h2[nx + 1] = val;
        if (xi == nx - 1) h2[0] = val;
    }
    __shared__ double sh[256];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = sh[0];
}

// Bias-gradient partials from a row-planar gradient: block (b, kc) sums the cells
// (slots 1 .. nx, not the halo copies) of plane kc of rows b, b + G, ... into
// bpart[(kc * G + b) * 8 + c], channel 8 kc + c.  A thread sums its values in
// binary32 (a few dozen terms), the block its threads' sums in binary64, in a
// fixed order.  Threads: 32 slots of a row x 8 rows at a time.
__global__ void bias_grad_rp_kernel(const bf16 *__restrict__ zn, int kcs, int nx, long long rows,
                                    double *__restrict__ bpart) {
    const int nxp = tc::rp_cells(nx);
    const int kc = blockIdx.y, G = gridDim.x;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    float s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (long long r = blockIdx.x + (long long)ty * G; r < rows; r += 8LL * G) {
        const uint4 *row = reinterpret_cast<const uint4 *>(zn + (r * kcs + kc) * nxp * 8);
        for (int j = 1 + tx; j <= nx; j += 32) {
            __align__(16) bf16 v[8];
            *reinterpret_cast<uint4 *>(v) = row[j];
#pragma unroll
            for (int c = 0; c < 8; ++c) s[c] += __bfloat162float(v[c]);
        }
    }
    __shared__ double sh[8][256];
#pragma unroll
    for (int c = 0; c < 8; ++c) sh[c][threadIdx.x] = (double)s[c];
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
#pragma unroll
            for (int c = 0; c < 8; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x < 8) bpart[((long long)kc * G + blockIdx.x) * 8 + threadIdx.x] = sh[threadIdx.x][0];
}

// gb[co] = sum over blocks of the partials above: one warp per channel, lane l
// taking blocks l, l + 32, ..., then a fixed shuffle tree.
__global__ void bias_reduce_kernel(const double *__restrict__ bpart, int G, float *__restrict__ gb) {
    const int co = blockIdx.x, lane = threadIdx.x;
    double s = 0.0;
    for (int b = lane; b < G; b += 32) s += bpart[((long long)(co / 8) * G + b) * 8 + co % 8];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) gb[co] = (float)s;
}

// Weights of the input-gradient convolution: Wt[ci][co][26 - tap] = W[co][ci][tap]
// (the adjoint of a cross-correlation correlates with the flipped kernel, input
// and output channels exchanged).
__global__ void flip_transpose_kernel(const float *__restrict__ W, int cout, int cin,
                                      float *__restrict__ Wt) {
    const int total = cout * cin * 27;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const int co = t / (cin * 27);
        const int rem = t - co * cin * 27;
        const int ci = rem / 27;
        const int tap = rem - ci * 27;
        Wt[((long long)ci * cout + co) * 27 + 26 - tap] = W[t];
    }
}

}  // namespace ac

using namespace ac;

// Parameter layout (binary32, as in common deep-learning libraries):
// W1[32][8][3][3][3], b1[32], W2[32][32][3][3][3], b2[32], W3[8][32][3][3][3], b3[8].
static const int P_W1 = 0, P_B1 = 6912, P_W2 = 6944, P_B2 = 34592, P_W3 = 34624, P_B3 = 41536;

struct ac_closure {
    ConvGeom g;
    cudaStream_t stream;
    float *block;  // master params, m, v, grads, scales
    float *params, *adam_m, *adam_v, *grads;
    float *scales;  // [0..7] 1/in_scale, [8..15] out_scale, [16..23] 1/out_scale
    float in_scale[8], out_scale[8];
    bf16 *wf1, *wf2, *wf3, *wb3, *wb2;
    bf16 *x0, *a1, *a2, *dy, *dz2, *dz1;
    float *y;
    // tcgen05 forward: weight images, tensor maps of the row-planar inputs of the
    // three layers (x0, a1, a2 hold the row-planar activations on this path)
    int conv_path;
    bf16 *img1, *img2, *img3;
    unsigned *tc_err;
    int tc_grid[3];
    int tc_zc;
    CUtensorMap tc_map[3];
    // paired-CTA forward: the two halves of each layer's kz stack, grid, segment length
    bf16 *pimg1, *pimg2, *pimg3;
    int tp_grid[3];
    int tp_smem[3];  // dynamic shared memory of a launch (at least half an SM's)
    int tp_zc;
    // tcgen05 training (allocated by the first backward pass on that path):
    // input-gradient weight images, gradients row-planar with halo (h, inputs of
    // the input-gradient convolutions) and without (n, weight-gradient operands),
    // tensor maps, per-CTA weight-gradient and bias partials
    void *train_block;
    bf16 *img3b, *img2b, *dyh, *dy2h, *dz2h, *dz1h;
    float *wt;      // flipped, transposed master weights of layers 3 and 2
    float *wpart;
    double *bpart;
    CUtensorMap tr_map[4];  // dyh, dz2h, dy2h, dz1h
    int tr_grid[5];         // conv<8,32,mask>, conv<32,32,mask>, wgrad<32,8>, <32,32>, <8,32>
    int tr_bias_blocks;
    float *part;
    double *lossp;
    double *loss_host;
    unsigned long long *guard;
    int adam_t;
    int lossblocks;
    unsigned long long launches;
    void *act_block;
};

#define CCK(call)                                          \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return ac_report_cuda(e_);  \
    } while (0)

static unsigned cl_grid(long long count, int threads = 256) {
    long long b = (count + threads - 1) / threads;
    return (unsigned)(b > 152 * 16 ? 152 * 16 : (b < 1 ? 1 : b));
}

template <int CIN, int COUT, int EPI>
static cudaError_t tc_grid_for(const ac_closure *c, int sms, int *grid) {
    auto k = tc::conv_tc_kernel<CIN, COUT, EPI>;
    const int bytes = (int)tc::smem_bytes(CIN, COUT < 16 ? 16 : COUT);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    int per_sm = 0;
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, tc::THREADS, bytes);
    if (e != cudaSuccess) return e;
    // an SM's 512 TMEM columns bound the resident CTAs too (each allocates RBLK blocks)
    const int tcols = tc::RBLK * (COUT < 16 ? 16 : COUT);
    if (per_sm > 512 / tcols) per_sm = 512 / tcols;
    const long long segs = (long long)((c->g.nz + c->tc_zc - 1) / c->tc_zc) * c->g.ny *
                           ((c->g.nx + tc::TM - 1) / tc::TM);
    long long g = (long long)(per_sm < 1 ? 1 : per_sm) * sms;
    *grid = (int)(g < segs ? g : segs);
    return cudaSuccess;
}

// Persistent grid of the paired kernel: as many CTA pairs as can be resident at
// once (clusters must fit within a GPC, so this can be below half the SMs),
// at most one per pair segment.  Each CTA allocates all 512 TMEM columns, so a
// second CTA on an SM would only wait for the first: the launch asks for more
// than half an SM's shared memory, which keeps it to one CTA per SM.
template <int CIN, int COUT, int EPI>
static cudaError_t tp_grid_for(const ac_closure *c, int sms, int *grid, int *smem) {
    auto k = tc::conv_tc_pair_kernel<CIN, COUT, EPI>;
    int dev = 0, per_sm_bytes = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&per_sm_bytes, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e != cudaSuccess) return e;
    int bytes = (int)tc::pair_smem_bytes(CIN);
    if (bytes < per_sm_bytes / 2 + 1024) bytes = per_sm_bytes / 2 + 1024;
    *smem = bytes;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(sms / 2 * 2), 1, 1);
    cfg.blockDim = dim3(tc::THREADS, 1, 1);
    cfg.dynamicSmemBytes = (size_t)bytes;
    cfg.stream = c->stream;
    int clusters = 0;
    e = cudaOccupancyMaxActiveClusters(&clusters, (const void *)k, &cfg);
    if (e != cudaSuccess) return e;
    const long long cols = (long long)c->g.ny * ((c->g.nx + tc::TM - 1) / tc::TM);
    const long long psegs = (long long)((c->g.nz + c->tp_zc - 1) / c->tp_zc) * ((cols + 1) / 2);
    long long n = clusters < 1 ? 1 : clusters;
    n = n < psegs ? n : psegs;
    *grid = (int)(2 * n);
    return cudaSuccess;
}

// Segment length of the paired kernel: every segment has the same length L <=
// PZC (the last z-chunk overlaps the one before); L minimises the slices staged
// per column, ceil(nz / L) (L + 2), the larger L on ties.
static int pair_zc(int nz) {
    int best = 1;
    long long cost = -1;
    for (int L = 1; L <= tc::PZC && L <= nz; ++L) {
        const long long k = (long long)((nz + L - 1) / L) * (L + 2);
        if (cost < 0 || k <= cost) {
            best = L;
            cost = k;
        }
    }
    return best;
}

// Tensor map of a row-planar activation with KC groups of 8 channels: dims
// (64 = 8 cells x 8 channels, nxp / 8, KC, ny, nz), box (64, 17, KC, 1, 1).
static cudaError_t tc_encode(PFN_cuTensorMapEncodeTiled_v12000 enc, const ac_closure *c, void *base,
                             int kc, CUtensorMap *map) {
    const cuuint64_t nxp = (cuuint64_t)tc::rp_cells(c->g.nx);
    const cuuint64_t dims[5] = {64, nxp / 8, (cuuint64_t)kc, (cuuint64_t)c->g.ny, (cuuint64_t)c->g.nz};
    const cuuint64_t strides[4] = {128, 16 * nxp, 16 * nxp * kc, 16 * nxp * kc * c->g.ny};
    const cuuint32_t box[5] = {64, tc::PCELLS / 8, (cuuint32_t)kc, 1, 1};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, base, dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Dynamic shared memory limits, persistent grid sizes and tensor maps of the
// three layers.
static cudaError_t tc_setup(ac_closure *c) {
    int dev = 0, sms = 0;
    c->tc_zc = c->g.nz < tc::RBLK ? c->g.nz : tc::RBLK;  // a segment fits the TMEM blocks
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = tc_grid_for<8, 32, tc::EPI_RELU_BF16>(c, sms, &c->tc_grid[0]);
    if (e == cudaSuccess) e = tc_grid_for<32, 32, tc::EPI_RELU_BF16>(c, sms, &c->tc_grid[1]);
    if (e == cudaSuccess) e = tc_grid_for<32, 8, tc::EPI_SCALED_F32>(c, sms, &c->tc_grid[2]);
    c->tp_zc = pair_zc(c->g.nz);
    if (e == cudaSuccess)
        e = tp_grid_for<8, 32, tc::EPI_RELU_BF16>(c, sms, &c->tp_grid[0], &c->tp_smem[0]);
    if (e == cudaSuccess)
        e = tp_grid_for<32, 32, tc::EPI_RELU_BF16>(c, sms, &c->tp_grid[1], &c->tp_smem[1]);
    if (e == cudaSuccess)
        e = tp_grid_for<32, 8, tc::EPI_SCALED_F32>(c, sms, &c->tp_grid[2], &c->tp_smem[2]);
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (e == cudaSuccess)
        e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e == cudaSuccess && (q != cudaDriverEntryPointSuccess || !fn)) e = cudaErrorNotSupported;
    if (e != cudaSuccess) return e;
    auto enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    e = tc_encode(enc, c, c->x0, 1, &c->tc_map[0]);
    if (e == cudaSuccess) e = tc_encode(enc, c, c->a1, 4, &c->tc_map[1]);
    if (e == cudaSuccess) e = tc_encode(enc, c, c->a2, 4, &c->tc_map[2]);
    return e;
}

static void free_closure(ac_closure *c) {
    if (c->block) cudaFree(c->block);
    if (c->act_block) cudaFree(c->act_block);
    if (c->train_block) cudaFree(c->train_block);
    if (c->loss_host) cudaFreeHost(c->loss_host);
}

extern "C" int ac_closure_init(ac_closure **out, int nx, int ny, int nz, void *stream) {
    if (!out || nx < 1 || ny < 1 || nz < 1 || nx > (1 << 20) || ny > (1 << 20) || nz > (1 << 20))
        return AC_ERR_ARG;
    *out = nullptr;
    ac_closure *c = new (std::nothrow) ac_closure();
    if (!c) return AC_ERR_OOM;
    c->g.nx = nx;
    c->g.ny = ny;
    c->g.nz = nz;
    c->g.n = (long long)nx * ny * nz;
    c->stream = static_cast<cudaStream_t>(stream);
    const long long n = c->g.n;
    const size_t np = AC_CLOSURE_NPARAMS;
    // params, m, v, grads, scales (24), bf16 weights (fwd and transposed layouts)
    const size_t wbytes = 2 * (32 * 27 * 16 + 32 * 27 * 32 + 8 * 27 * 32 + 32 * 27 * 16 + 32 * 27 * 32) +
                          2 * (27 * 16 * 32 + 27 * 32 * 32 + 27 * 32 * 16) +
                          (size_t)tc::w_bytes(8, 32) + 2 * (size_t)tc::w_bytes(32, 32);
    const size_t fbytes = sizeof(float) * (4 * np + 64) + wbytes + 256;
    c->lossblocks = 304;
    const size_t part_floats = (size_t)9 * CL_WG_CTAS * 32 * 96;
    // x0, a1, a2 hold either channel-major [C][n] or row-planar [rows][C/8][nx+2][8]
    // activations: sized for the larger (row-planar, np2 cells per channel)
    const long long np2 = (long long)tc::rp_cells(nx) * ny * nz;
    const size_t abytes = 2 * (size_t)np2 * (16 + 32 + 32) + 2 * (size_t)n * (16 + 32 + 32) +
                          4 * (size_t)n * 8 + 4 * part_floats + 8 * (size_t)c->lossblocks + 8 + 1024;
    cudaError_t e = cudaMalloc(&c->block, fbytes);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->block, 0, fbytes, c->stream);
    if (e == cudaSuccess) e = cudaMalloc(&c->act_block, abytes);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->act_block, 0, abytes, c->stream);
    if (e == cudaSuccess) e = cudaMallocHost(&c->loss_host, 2 * sizeof(double));
    if (e != cudaSuccess) {
        int rc = ac_report_cuda(e);
        free_closure(c);
        delete c;
        return rc;
    }
    float *f = c->block;
    c->params = f;
    c->adam_m = f + np;
    c->adam_v = f + 2 * np;
    c->grads = f + 3 * np;
    c->scales = f + 4 * np;
    bf16 *w = reinterpret_cast<bf16 *>(f + 4 * np + 64);
    c->wf1 = w;
    c->wf2 = c->wf1 + 32 * 27 * 16;
    c->wf3 = c->wf2 + 32 * 27 * 32;
    c->wb3 = c->wf3 + 8 * 27 * 32;
    c->wb2 = c->wb3 + 32 * 27 * 16;
    c->img1 = c->wb2 + 32 * 27 * 32;  // byte offsets stay multiples of 16
    c->img2 = c->img1 + 27 * 16 * 32;
    c->img3 = c->img2 + 27 * 32 * 32;
    c->pimg1 = c->img3 + 27 * 32 * 16;
    c->pimg2 = c->pimg1 + tc::w_bytes(8, 32) / 2;
    c->pimg3 = c->pimg2 + tc::w_bytes(32, 32) / 2;
    char *a = static_cast<char *>(c->act_block);
    c->x0 = reinterpret_cast<bf16 *>(a);
    c->a1 = c->x0 + 16 * np2;
    c->a2 = c->a1 + 32 * np2;
    c->dy = c->a2 + 32 * np2;
    c->dz2 = c->dy + 16 * n;
    c->dz1 = c->dz2 + 32 * n;
    c->y = reinterpret_cast<float *>(c->dz1 + 32 * n);
    c->part = c->y + 8 * n;
    c->lossp = reinterpret_cast<double *>(c->part + part_floats);
    c->guard = reinterpret_cast<unsigned long long *>(c->lossp + c->lossblocks);
    c->tc_err = reinterpret_cast<unsigned *>(c->guard + 1);
    for (int i = 0; i < 8; ++i) c->in_scale[i] = c->out_scale[i] = 1.f;
    float sc[32];  // [24..31]: ones, the output scale of the training forward pass
    for (int i = 0; i < 32; ++i) sc[i] = 1.f;
    e = cudaMemcpyAsync(c->scales, sc, sizeof sc, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) e = tc_setup(c);
    if (e != cudaSuccess) {
        int rc = ac_report_cuda(e);
        free_closure(c);
        delete c;
        return rc;
    }
    *out = c;
    return AC_OK;
}

extern "C" int ac_closure_quit(ac_closure *c) {
    if (!c) return AC_OK;
    cudaStreamSynchronize(c->stream);
    free_closure(c);
    delete c;
    return AC_OK;
}

// Input-gradient weight images of layers 3 and 2 (the tcgen05 training path):
// the flipped, transposed weights in the image order of conv_tc_kernel.
static void prep_train_images(ac_closure *c) {
    float *wt3 = c->wt, *wt2 = c->wt + 8 * 32 * 27;
    flip_transpose_kernel<<<32, 256, 0, c->stream>>>(c->params + P_W3, 8, 32, wt3);
    flip_transpose_kernel<<<128, 256, 0, c->stream>>>(c->params + P_W2, 32, 32, wt2);
    tc::conv_tc_prep_kernel<<<16, 256, 0, c->stream>>>(wt3, 32, 8, 8, 32, 0, 12, c->img3b);
    tc::conv_tc_prep_kernel<<<128, 256, 0, c->stream>>>(wt2, 32, 32, 32, 32, 0, 12, c->img2b);
    c->launches += 4;
}

static int prep_weights(ac_closure *c) {
    if (c->train_block) prep_train_images(c);
    prep_weights_kernel<<<32, 256, 0, c->stream>>>(c->params + P_W1, 32, 8, 16, c->wf1, 0, nullptr);
    prep_weights_kernel<<<128, 256, 0, c->stream>>>(c->params + P_W2, 32, 32, 32, c->wf2, 32, c->wb2);
    prep_weights_kernel<<<32, 256, 0, c->stream>>>(c->params + P_W3, 8, 32, 32, c->wf3, 16, c->wb3);
    tc::conv_tc_prep_kernel<<<16, 256, 0, c->stream>>>(c->params + P_W1, 32, 8, 8, 32, 0, 12, c->img1);
    tc::conv_tc_prep_kernel<<<128, 256, 0, c->stream>>>(c->params + P_W2, 32, 32, 32, 32, 0, 12,
                                                        c->img2);
    tc::conv_tc_prep_kernel<<<64, 256, 0, c->stream>>>(c->params + P_W3, 8, 32, 32, 16, 0, 6, c->img3);
    // paired kernel: stack rows 0..47 (core rows 0..5) then 48..95, 32 per kz
    for (int h = 0; h < 2; ++h) {
        tc::conv_tc_prep_kernel<<<16, 256, 0, c->stream>>>(c->params + P_W1, 32, 8, 8, 32, 6 * h, 6,
                                                           c->pimg1 + h * tc::w_bytes(8, 32) / 4);
        tc::conv_tc_prep_kernel<<<64, 256, 0, c->stream>>>(c->params + P_W2, 32, 32, 32, 32, 6 * h, 6,
                                                           c->pimg2 + h * tc::w_bytes(32, 32) / 4);
        tc::conv_tc_prep_kernel<<<64, 256, 0, c->stream>>>(c->params + P_W3, 8, 32, 32, 32, 6 * h, 6,
                                                           c->pimg3 + h * tc::w_bytes(32, 32) / 4);
    }
    c->launches += 12;
    CCK(cudaGetLastError());
    return AC_OK;
}

extern "C" int ac_closure_set_params(ac_closure *c, const float *host) {
    if (!c || !host) return AC_ERR_ARG;
    for (int i = 0; i < AC_CLOSURE_NPARAMS; ++i)
        if (!isfinite(host[i])) return AC_ERR_ARG;
    CCK(cudaMemcpyAsync(c->params, host, sizeof(float) * AC_CLOSURE_NPARAMS, cudaMemcpyHostToDevice,
                        c->stream));
    CCK(cudaMemsetAsync(c->adam_m, 0, sizeof(float) * 2 * AC_CLOSURE_NPARAMS, c->stream));
    c->adam_t = 0;
    return prep_weights(c);
}

static int copy_out(ac_closure *c, const float *dev, float *host) {
    if (!c || !host) return AC_ERR_ARG;
    CCK(cudaMemcpyAsync(host, dev, sizeof(float) * AC_CLOSURE_NPARAMS, cudaMemcpyDeviceToHost,
                        c->stream));
    CCK(cudaStreamSynchronize(c->stream));
    return AC_OK;
}

extern "C" int ac_closure_get_params(ac_closure *c, float *host) {
    return c ? copy_out(c, c->params, host) : AC_ERR_ARG;
}
extern "C" int ac_closure_get_grads(ac_closure *c, float *host) {
    return c ? copy_out(c, c->grads, host) : AC_ERR_ARG;
}

extern "C" int ac_closure_set_scales(ac_closure *c, const float in_scale[8], const float out_scale[8]) {
    if (!c || !in_scale || !out_scale) return AC_ERR_ARG;
    float sc[24];
    for (int i = 0; i < 8; ++i) {
        if (!(in_scale[i] > 0) || !(out_scale[i] > 0) || !isfinite(in_scale[i]) ||
            !isfinite(out_scale[i]))
            return AC_ERR_ARG;
        c->in_scale[i] = in_scale[i];
        c->out_scale[i] = out_scale[i];
        sc[i] = 1.f / in_scale[i];
        sc[8 + i] = out_scale[i];
        sc[16 + i] = 1.f / out_scale[i];
    }
    CCK(cudaMemcpyAsync(c->scales, sc, sizeof sc, cudaMemcpyHostToDevice, c->stream));
    CCK(cudaStreamSynchronize(c->stream));
    return AC_OK;
}

// ev (optional): events recorded before the input pack and after the pack and
// each convolution launch (five of the six that ac_closure_forward_timings uses).
static inline void mark(cudaEvent_t *ev, int i, cudaStream_t st) {
    if (ev) cudaEventRecord(ev[i], st);
}

static int run_forward(ac_closure *c, const float *const in[8], cudaEvent_t *ev = nullptr) {
    const ConvGeom g = c->g;
    F8 f;
    for (int i = 0; i < 8; ++i) f.p[i] = in[i];
    mark(ev, 0, c->stream);
    pack_input_kernel<<<cl_grid(16 * g.n), 256, 0, c->stream>>>(f, c->scales, g.n, c->x0);
    mark(ev, 1, c->stream);
    const unsigned ctas = (unsigned)((long long)g.ny * g.nz * ((g.nx + CL_TM - 1) / CL_TM));
    conv_fwd_kernel<16, 32, EPI_RELU_BF16><<<ctas, CL_THREADS, 0, c->stream>>>(
        c->x0, c->wf1, c->params + P_B1, nullptr, c->a1, g);
    mark(ev, 2, c->stream);
    conv_fwd_kernel<32, 32, EPI_RELU_BF16><<<ctas, CL_THREADS, 0, c->stream>>>(
        c->a1, c->wf2, c->params + P_B2, nullptr, c->a2, g);
    mark(ev, 3, c->stream);
    conv_fwd_kernel<32, 8, EPI_LINEAR_F32><<<ctas, CL_THREADS, 0, c->stream>>>(
        c->a2, c->wf3, c->params + P_B3, nullptr, c->y, g);
    mark(ev, 4, c->stream);
    c->launches += 4;
    CCK(cudaGetLastError());
    return AC_OK;
}

// One layer on the tcgen05 kernels: the single-CTA kernel with the whole kz
// stack (img), or, when pair is set, the paired kernel with the two stack halves
// (pimg).
template <int CIN, int COUT, int EPI>
static void launch_tc(const ac_closure *c, int layer, bool pair, const bf16 *img, const bf16 *pimg,
                      const float *bias, bf16 *y, float *const out[8] = nullptr,
                      unsigned long long *gmax = nullptr, const float *oscale = nullptr) {
    tc::ConvTcArgs a;
    a.w = img;
    a.bias = bias;
    a.y = y;
    a.mask = nullptr;
    for (int i = 0; i < 8; ++i) a.out[i] = out ? out[i] : nullptr;
    a.out_scale = oscale ? oscale : c->scales + 8;
    a.gmax = gmax;
    a.nx = c->g.nx;
    a.ny = c->g.ny;
    a.nz = c->g.nz;
    a.zc = pair ? c->tp_zc : c->tc_zc;
    a.err = c->tc_err;
    if (pair) {
        a.w = pimg;
        tc::conv_tc_pair_kernel<CIN, COUT, EPI>
            <<<c->tp_grid[layer], tc::THREADS, c->tp_smem[layer], c->stream>>>(c->tc_map[layer], a);
        return;
    }
    tc::conv_tc_kernel<CIN, COUT, EPI>
        <<<c->tc_grid[layer], tc::THREADS, tc::smem_bytes(CIN, COUT < 16 ? 16 : COUT), c->stream>>>(
            c->tc_map[layer], a);
}

// Forward pass on the tcgen05 kernels (row-planar activations in x0, a1, a2);
// layer 3 writes out_scale * net(...) channel-major to out[0..7] (the closure's
// own y when out is null) and, if gmax is given, folds the largest |value| into it.
// With unscaled set, layer 3 writes net(...) itself (training).
static int run_forward_tc(ac_closure *c, const float *const in[8], float *const out[8],
                          unsigned long long *gmax, cudaEvent_t *ev = nullptr,
                          bool unscaled = false) {
    const ConvGeom g = c->g;
    F8 f;
    for (int i = 0; i < 8; ++i) f.p[i] = in[i];
    float *own[8];
    for (int i = 0; i < 8; ++i) own[i] = c->y + (long long)i * g.n;
    mark(ev, 0, c->stream);
    pack_input_rp_kernel<<<cl_grid(g.n), 256, 0, c->stream>>>(f, c->scales, g.nx, g.n, c->x0);
    mark(ev, 1, c->stream);
    const bool pair = c->conv_path == AC_CONV_TCGEN05_PAIR;
    launch_tc<8, 32, tc::EPI_RELU_BF16>(c, 0, pair, c->img1, c->pimg1, c->params + P_B1, c->a1);
    mark(ev, 2, c->stream);
    launch_tc<32, 32, tc::EPI_RELU_BF16>(c, 1, pair, c->img2, c->pimg2, c->params + P_B2, c->a2);
    mark(ev, 3, c->stream);
    launch_tc<32, 8, tc::EPI_SCALED_F32>(c, 2, pair, c->img3, c->pimg3, c->params + P_B3, nullptr,
                                         out ? out : own, gmax, unscaled ? c->scales + 24 : nullptr);
    mark(ev, 4, c->stream);
    c->launches += 4;
    CCK(cudaGetLastError());
    return AC_OK;
}

// Inference on the selected path: the scaled correction in out (or the closure's
// own y when null); ev, if given, brackets the five launches of the mma.sync path
// (on the tcgen05 path the fifth, the output scaling, is empty).
static int run_inference(ac_closure *c, const float *const in[8], float *const out[8],
                         cudaEvent_t *ev = nullptr) {
    if (c->conv_path != AC_CONV_MMA_SYNC) {
        int rc = run_forward_tc(c, in, out, nullptr, ev);
        mark(ev, 5, c->stream);
        return rc;
    }
    int rc = run_forward(c, in, ev);
    if (rc == AC_OK && out) {
        W8 o;
        for (int i = 0; i < 8; ++i) o.p[i] = out[i];
        scale_output_kernel<<<cl_grid(8 * c->g.n), 256, 0, c->stream>>>(c->y, c->scales + 8, c->g.n, o);
        c->launches++;
        CCK(cudaGetLastError());
    }
    mark(ev, 5, c->stream);
    return rc;
}

extern "C" int ac_closure_set_conv_path(ac_closure *c, int path) {
    if (!c || (path != AC_CONV_TCGEN05 && path != AC_CONV_MMA_SYNC && path != AC_CONV_TCGEN05_PAIR))
        return AC_ERR_ARG;
    c->conv_path = path;
    return AC_OK;
}

extern "C" int ac_closure_get_conv_path(const ac_closure *c, int *path) {
    if (!c || !path) return AC_ERR_ARG;
    *path = c->conv_path;
    return AC_OK;
}

extern "C" int ac_closure_status(ac_closure *c) {
    if (!c) return AC_ERR_ARG;
    unsigned err = 0;
    CCK(cudaMemcpyAsync(c->loss_host, c->tc_err, sizeof err, cudaMemcpyDeviceToHost, c->stream));
    CCK(cudaMemsetAsync(c->tc_err, 0, sizeof err, c->stream));
    CCK(cudaStreamSynchronize(c->stream));
    memcpy(&err, c->loss_host, sizeof err);
    return err ? AC_ERR_TIMEOUT : AC_OK;
}

extern "C" int ac_diag_wait_timeout(unsigned polls, void *stream) {
    if (polls == 0 || polls > tc::WAIT_LIMIT) return AC_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned *d = nullptr;
    unsigned h = 2;
    cudaError_t e = cudaMalloc(&d, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemsetAsync(d, 0xff, sizeof(unsigned), st);
    if (e == cudaSuccess) {
        tc::wait_timeout_kernel<<<1, 32, 0, st>>>(polls, d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof h, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (d) cudaFree(d);
    if (e != cudaSuccess) return ac_report_cuda(e);
    return h == 1u ? AC_ERR_TIMEOUT : (h == 0u ? AC_OK : AC_ERR_CUDA);
}

extern "C" int ac_closure_forward(ac_closure *c, const float *const in[8], float *const out[8]) {
    AC_RANGE("ac_closure_forward");
    if (!c || !in) return AC_ERR_ARG;
    for (int i = 0; i < 8; ++i)
        if (!in[i] || (out && !out[i])) return AC_ERR_ARG;
    return run_inference(c, in, out);
}

extern "C" int ac_closure_forward_timings(ac_closure *c, const float *const in[8],
                                          float *const out[8], float ms[5]) {
    if (!c || !in || !out || !ms) return AC_ERR_ARG;
    for (int i = 0; i < 8; ++i)
        if (!in[i] || !out[i]) return AC_ERR_ARG;
    cudaEvent_t ev[6] = {};
    int rc = AC_OK;
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 6 && e == cudaSuccess; ++i) e = cudaEventCreate(&ev[i]);
    if (e == cudaSuccess) {
        rc = run_inference(c, in, out, ev);
        if (rc == AC_OK) {
            e = cudaEventSynchronize(ev[5]);
            for (int i = 0; i < 5 && e == cudaSuccess; ++i) e = cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]);
        }
    }
    for (int i = 0; i < 6; ++i)
        if (ev[i]) cudaEventDestroy(ev[i]);
    if (rc == AC_OK && e != cudaSuccess) rc = ac_report_cuda(e);
    return rc;
}

// Mean squared error from the loss kernel's block partials (waits for the stream).
static int read_loss(ac_closure *c, double *loss) {
    double *hp = static_cast<double *>(malloc(sizeof(double) * c->lossblocks));
    if (!hp) return AC_ERR_OOM;
    cudaError_t e = cudaMemcpyAsync(hp, c->lossp, sizeof(double) * c->lossblocks,
                                    cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        free(hp);
        return ac_report_cuda(e);
    }
    double s = 0.0;
    for (int i = 0; i < c->lossblocks; ++i) s += hp[i];
    free(hp);
    *loss = s / (8.0 * (double)c->g.n);
    return isfinite(*loss) ? AC_OK : AC_ERR_NONFINITE;
}

// Persistent grid of a weight-gradient kernel: resident CTAs (shared memory and
// an SM's 512 TMEM columns bound them) times SMs, at most one per segment.
template <int CIN, int COUT>
static cudaError_t wgrad_grid_for(const ac_closure *c, int sms, int *grid) {
    using S = tc::WgradShape<CIN, COUT>;
    auto k = tc::wgrad_tc_kernel<CIN, COUT>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
    int per_sm = 0;
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, tc::THREADS, S::SMEM);
    if (e != cudaSuccess) return e;
    if (per_sm > 512 / S::TCOLS) per_sm = 512 / S::TCOLS;
    const long long segs = (long long)((c->g.nz + c->tc_zc - 1) / c->tc_zc) * c->g.ny *
                           ((c->g.nx + tc::TM - 1) / tc::TM);
    long long g = (long long)(per_sm < 1 ? 1 : per_sm) * sms;
    *grid = (int)(g < segs ? g : segs);
    return cudaSuccess;
}

static size_t align256(size_t b) { return (b + 255) / 256 * 256; }

// Buffers, tensor maps, grids and weight images of the tcgen05 training path,
// made by its first backward pass.
static int ensure_train(ac_closure *c) {
    if (c->train_block) return AC_OK;
    int dev = 0, sms = 0;
    CCK(cudaGetDevice(&dev));
    CCK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CCK((tc_grid_for<8, 32, tc::EPI_MASK_BF16>(c, sms, &c->tr_grid[0])));
    CCK((tc_grid_for<32, 32, tc::EPI_MASK_BF16>(c, sms, &c->tr_grid[1])));
    CCK((wgrad_grid_for<32, 8>(c, sms, &c->tr_grid[2])));
    CCK((wgrad_grid_for<32, 32>(c, sms, &c->tr_grid[3])));
    CCK((wgrad_grid_for<8, 32>(c, sms, &c->tr_grid[4])));
    int wmax = 0;  // largest per-CTA partial block (floats) times grid
    {
        const int per[3] = {tc::WgradShape<32, 8>::NACC * tc::WgradShape<32, 8>::N3,
                            tc::WgradShape<32, 32>::NACC * tc::WgradShape<32, 32>::N3,
                            tc::WgradShape<8, 32>::NACC * tc::WgradShape<8, 32>::N3};
        for (int l = 0; l < 3; ++l)
            if (per[l] * c->tr_grid[2 + l] > wmax) wmax = per[l] * c->tr_grid[2 + l];
    }
    const long long rows = (long long)c->g.ny * c->g.nz;
    // bias partial blocks: about 64 rows each (a thread's binary32 sum stays short)
    c->tr_bias_blocks = (int)(rows / 64 < 1 ? 1 : (rows / 64 > 4096 ? 4096 : rows / 64));
    const long long np2 = (long long)tc::rp_cells(c->g.nx) * rows;
    const size_t b_wpart = align256(sizeof(float) * (size_t)wmax * tc::TM);
    const size_t b_bpart = align256(sizeof(double) * 4 * (size_t)c->tr_bias_blocks * 8);
    const size_t b_wt = align256(sizeof(float) * (8 * 32 * 27 + 32 * 32 * 27));
    const size_t b_img3 = align256((size_t)tc::w_bytes(8, 32));
    const size_t b_img2 = align256((size_t)tc::w_bytes(32, 32));
    // dyh (8 channels), dy2h (16: 8 and a zero plane), dz2h, dz1h (32), row-planar with halo
    const size_t b_act[4] = {align256(2 * 8 * (size_t)np2), align256(2 * 16 * (size_t)np2),
                             align256(2 * 32 * (size_t)np2), align256(2 * 32 * (size_t)np2)};
    size_t total = b_wpart + b_bpart + b_wt + b_img3 + b_img2;
    for (int i = 0; i < 4; ++i) total += b_act[i];
    void *blk = nullptr;
    cudaError_t e = cudaMalloc(&blk, total);
    if (e == cudaSuccess) e = cudaMemsetAsync(blk, 0, total, c->stream);  // zero halos and padding
    if (e != cudaSuccess) {
        if (blk) cudaFree(blk);
        return ac_report_cuda(e);
    }
    char *p = static_cast<char *>(blk);
    c->wpart = reinterpret_cast<float *>(p);
    p += b_wpart;
    c->bpart = reinterpret_cast<double *>(p);
    p += b_bpart;
    c->wt = reinterpret_cast<float *>(p);
    p += b_wt;
    c->img3b = reinterpret_cast<bf16 *>(p);
    p += b_img3;
    c->img2b = reinterpret_cast<bf16 *>(p);
    p += b_img2;
    bf16 **acts[4] = {&c->dyh, &c->dy2h, &c->dz2h, &c->dz1h};
    for (int i = 0; i < 4; ++i) {
        *acts[i] = reinterpret_cast<bf16 *>(p);
        p += b_act[i];
    }
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e == cudaSuccess && (q != cudaDriverEntryPointSuccess || !fn)) e = cudaErrorNotSupported;
    auto enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    const int kcs[4] = {1, 4, 2, 4};
    bf16 *bases[4] = {c->dyh, c->dz2h, c->dy2h, c->dz1h};
    for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = tc_encode(enc, c, bases[i], kcs[i], &c->tr_map[i]);
    if (e != cudaSuccess) {
        cudaFree(blk);
        return ac_report_cuda(e);
    }
    c->train_block = blk;
    prep_train_images(c);
    CCK(cudaGetLastError());
    return AC_OK;
}

// One input-gradient convolution through a ReLU on the tcgen05 kernel: from the
// row-planar gradient behind xmap, with image img, mask = the forward activation;
// writes y (with its halo cells).
template <int CIN>
static void launch_mask(const ac_closure *c, const CUtensorMap &xmap, int grid, const bf16 *img,
                        const bf16 *mask, bf16 *y) {
    tc::ConvTcArgs a = {};
    a.w = img;
    a.y = y;
    a.mask = mask;
    a.nx = c->g.nx;
    a.ny = c->g.ny;
    a.nz = c->g.nz;
    a.zc = c->tc_zc;
    a.err = c->tc_err;
    tc::conv_tc_kernel<CIN, 32, tc::EPI_MASK_BF16>
        <<<grid, tc::THREADS, tc::smem_bytes(CIN, 32), c->stream>>>(xmap, a);
}

template <int CIN, int COUT>
static void launch_wgrad(const ac_closure *c, const CUtensorMap &xmap, const CUtensorMap &dmap,
                         int grid, int cin_real, float *gW) {
    tc::WgradTcArgs a;
    a.part = c->wpart;
    a.nx = c->g.nx;
    a.ny = c->g.ny;
    a.nz = c->g.nz;
    a.zc = c->tc_zc;
    a.err = c->tc_err;
    tc::wgrad_tc_kernel<CIN, COUT>
        <<<grid, tc::THREADS, tc::WgradShape<CIN, COUT>::SMEM, c->stream>>>(xmap, dmap, a);
    tc::wgrad_tc_reduce_kernel<CIN, COUT><<<152, 256, 0, c->stream>>>(c->wpart, grid, cin_real, gW);
}

static void launch_bias(const ac_closure *c, const bf16 *zn, int kcs, int cout, float *gb) {
    const long long rows = (long long)c->g.ny * c->g.nz;
    bias_grad_rp_kernel<<<dim3((unsigned)c->tr_bias_blocks, (unsigned)(cout / 8)), 256, 0, c->stream>>>(
        zn, kcs, c->g.nx, rows, c->bpart);
    bias_reduce_kernel<<<cout, 32, 0, c->stream>>>(c->bpart, c->tr_bias_blocks, gb);
}

// Backward pass on the tcgen05 kernels: forward (row-planar activations kept),
// loss and dY, the two input gradients through the ReLUs (flipped, transposed
// weights), the three weight gradients and the three bias gradients.
static int run_backward_tc(ac_closure *c, const float *const in[8], const float *const target[8]) {
    int rc = ensure_train(c);
    if (rc) return rc;
    rc = run_forward_tc(c, in, nullptr, nullptr, nullptr, true);
    if (rc) return rc;
    const ConvGeom g = c->g;
    F8 t;
    for (int i = 0; i < 8; ++i) t.p[i] = target[i];
    loss_grad_rp_kernel<<<c->lossblocks, 256, 0, c->stream>>>(c->y, t, c->scales + 16, g.nx, g.n,
                                                              c->dyh, c->dy2h, c->lossp);
    launch_mask<8>(c, c->tr_map[0], c->tr_grid[0], c->img3b, c->a2, c->dz2h);
    launch_mask<32>(c, c->tr_map[1], c->tr_grid[1], c->img2b, c->a1, c->dz1h);
    launch_wgrad<32, 8>(c, c->tc_map[2], c->tr_map[2], c->tr_grid[2], 32, c->grads + P_W3);
    launch_wgrad<32, 32>(c, c->tc_map[1], c->tr_map[1], c->tr_grid[3], 32, c->grads + P_W2);
    launch_wgrad<8, 32>(c, c->tc_map[0], c->tr_map[3], c->tr_grid[4], 8, c->grads + P_W1);
    launch_bias(c, c->dy2h, 2, 8, c->grads + P_B3);
    launch_bias(c, c->dz2h, 4, 32, c->grads + P_B2);
    launch_bias(c, c->dz1h, 4, 32, c->grads + P_B1);
    c->launches += 15;
    CCK(cudaGetLastError());
    return AC_OK;
}

extern "C" int ac_closure_backward(ac_closure *c, const float *const in[8],
                                   const float *const target[8], double *loss) {
    AC_RANGE("ac_closure_backward");
    if (!c || !in || !target) return AC_ERR_ARG;
    for (int i = 0; i < 8; ++i)
        if (!in[i] || !target[i]) return AC_ERR_ARG;
    const ConvGeom g = c->g;
    if (c->conv_path != AC_CONV_MMA_SYNC) {
        int rc = run_backward_tc(c, in, target);
        if (rc) return rc;
        return loss ? read_loss(c, loss) : AC_OK;
    }
    int rc = run_forward(c, in);
    if (rc) return rc;
    F8 t;
    for (int i = 0; i < 8; ++i) t.p[i] = target[i];
    loss_grad_kernel<<<c->lossblocks, 256, 0, c->stream>>>(c->y, t, c->scales + 16, g.n, c->dy,
                                                           c->lossp);
    const unsigned ctas = (unsigned)((long long)g.ny * g.nz * ((g.nx + CL_TM - 1) / CL_TM));
    // input gradients through conv3 and conv2 (ReLU masks from the stored activations)
    conv_fwd_kernel<16, 32, EPI_MASK_BF16><<<ctas, CL_THREADS, 0, c->stream>>>(
        c->dy, c->wb3, nullptr, c->a2, c->dz2, g);
    conv_fwd_kernel<32, 32, EPI_MASK_BF16><<<ctas, CL_THREADS, 0, c->stream>>>(
        c->dz2, c->wb2, nullptr, c->a1, c->dz1, g);
    // weight gradients
    const dim3 wg(CL_WG_CTAS, 9);
    conv_wgrad_kernel<32, 8><<<wg, CL_THREADS, 0, c->stream>>>(c->dy, c->a2, c->part, g);
    wgrad_reduce_kernel<<<32, 256, 0, c->stream>>>(c->part, CL_WG_CTAS, 8, 32, 32, c->grads + P_W3);
    conv_wgrad_kernel<32, 32><<<wg, CL_THREADS, 0, c->stream>>>(c->dz2, c->a1, c->part, g);
    wgrad_reduce_kernel<<<64, 256, 0, c->stream>>>(c->part, CL_WG_CTAS, 32, 32, 32, c->grads + P_W2);
    conv_wgrad_kernel<16, 32><<<wg, CL_THREADS, 0, c->stream>>>(c->dz1, c->x0, c->part, g);
    wgrad_reduce_kernel<<<32, 256, 0, c->stream>>>(c->part, CL_WG_CTAS, 32, 16, 8, c->grads + P_W1);
    bias_grad_kernel<<<8, 256, 0, c->stream>>>(c->dy, g.n, c->grads + P_B3);
    bias_grad_kernel<<<32, 256, 0, c->stream>>>(c->dz2, g.n, c->grads + P_B2);
    bias_grad_kernel<<<32, 256, 0, c->stream>>>(c->dz1, g.n, c->grads + P_B1);
    c->launches += 12;
    CCK(cudaGetLastError());
    return loss ? read_loss(c, loss) : AC_OK;
}

extern "C" int ac_closure_adam_step(ac_closure *c, float lr, float beta1, float beta2, float eps) {
    AC_RANGE("ac_closure_adam_step");
    if (!c || !(lr > 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) || !(eps > 0))
        return AC_ERR_ARG;
    c->adam_t++;
    const float c1 = 1.f - powf(beta1, (float)c->adam_t);
    const float c2 = 1.f - powf(beta2, (float)c->adam_t);
    adam_kernel<<<64, 256, 0, c->stream>>>(c->params, c->adam_m, c->adam_v, c->grads,
                                           AC_CLOSURE_NPARAMS, lr, beta1, beta2, eps, c1, c2);
    c->launches++;
    CCK(cudaGetLastError());
    return prep_weights(c);
}

extern "C" int ac_closure_apply(ac_closure *c, ac_handle *h, double limit, int *applied) {
    AC_RANGE("ac_closure_apply");
    if (!c || !h || !(limit > 0)) return AC_ERR_ARG;
    void *ptrs[8];
    int precision = 0, layout = 0, n[3];
    int rc = ac_get_state(h, ptrs, &precision, &layout, n);
    if (rc) return rc;
    if (precision == AC_FP64 || layout != AC_LAYOUT_PERIODIC || n[0] != c->g.nx ||
        n[1] != c->g.ny || n[2] != c->g.nz)
        return AC_ERR_ARG;
    const float *in[8];
    W8 f;
    for (int i = 0; i < 8; ++i) {
        in[i] = static_cast<const float *>(ptrs[i]);
        f.p[i] = static_cast<float *>(ptrs[i]);
    }
    CCK(cudaMemsetAsync(c->guard, 0, sizeof(unsigned long long), c->stream));
    const float *yscale = nullptr;  // y already scaled (tcgen05 path)
    if (c->conv_path != AC_CONV_MMA_SYNC) {
        rc = run_forward_tc(c, in, nullptr, c->guard);
        if (rc) return rc;
    } else {
        rc = run_forward(c, in);
        if (rc) return rc;
        correction_max_kernel<<<cl_grid(8 * c->g.n), 256, 0, c->stream>>>(c->y, c->scales + 8,
                                                                          c->g.n, c->guard);
        c->launches++;
        yscale = c->scales + 8;
    }
    apply_correction_kernel<<<cl_grid(8 * c->g.n), 256, 0, c->stream>>>(f, c->y, yscale, c->g.n,
                                                                        c->guard, limit);
    c->launches++;
    CCK(cudaGetLastError());
    if (applied) {
        unsigned long long bits = 0;
        CCK(cudaMemcpyAsync(c->loss_host, c->guard, sizeof bits, cudaMemcpyDeviceToHost, c->stream));
        CCK(cudaStreamSynchronize(c->stream));
        memcpy(&bits, c->loss_host, sizeof bits);
        double m;
        memcpy(&m, &bits, sizeof m);
        *applied = m <= limit ? 1 : 0;
    }
    return AC_OK;
}

extern "C" int ac_closure_launch_count(const ac_closure *c, unsigned long long *count) {
    if (!c || !count) return AC_ERR_ARG;
    *count = c->launches;
    return AC_OK;
}

extern "C" int ac_restrict(const void *const fine[8], int fine_precision, int nx, int ny, int nz,
                           float *const coarse[8], void *stream) {
    if (!fine || !coarse || nx < 2 || ny < 2 || nz < 2 || (nx | ny | nz) & 1) return AC_ERR_ARG;
    if (fine_precision != AC_FP64 && fine_precision != AC_FP32 && fine_precision != AC_FP32_W64)
        return AC_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const long long nc = (long long)(nx / 2) * (ny / 2) * (nz / 2);
    for (int q = 0; q < 8; ++q) {
        if (!fine[q] || !coarse[q]) return AC_ERR_ARG;
        if (fine_precision == AC_FP64)
            restrict_kernel<double><<<cl_grid(nc), 256, 0, st>>>(
                static_cast<const double *>(fine[q]), nx, ny, nz, coarse[q]);
        else
            restrict_kernel<float><<<cl_grid(nc), 256, 0, st>>>(
                static_cast<const float *>(fine[q]), nx, ny, nz, coarse[q]);
    }
    CCK(cudaGetLastError());
    return AC_OK;
}

AC_BC_READER(bc_take_closure)
