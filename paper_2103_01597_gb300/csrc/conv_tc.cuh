// 3-D convolution (3x3x3 taps, circular padding) as an implicit GEMM on the
// fifth-generation tensor cores: tcgen05.mma with bfloat16 operands from
// shared memory and a binary32 accumulator in tensor memory (TMEM).
//
// Activations are channels-last bfloat16, x[p][c] (p = cell, x fastest).  A CTA
// computes 128 cells of one x-row (GEMM M = 128) for all output channels
// (N = COUT, padded to 16).  K = 27 taps x CIN: for each tap, the 128 source
// cells (shifted by the tap, wrapped periodically) are copied with 16-byte
// cp.async into the canonical K-major no-swizzle layout (core matrices of
// 8 cells x 8 channels, 128 contiguous bytes), and one elected thread issues
// CIN/16 MMAs of K = 16.  A tiles are double-buffered: the copy of tap t+1
// overlaps the MMAs of tap t, and a buffer is refilled only after the MMAs
// that read it have signalled their mbarrier (tcgen05.commit).  The weights
// of the layer stay in shared memory in the same layout.  The epilogue reads
// the accumulator with tcgen05.ld (one row per thread) and applies bias and
// ReLU.  Every wait is bounded: on timeout the kernel records an error word,
// stops issuing, still frees its TMEM, and returns.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace ac {
namespace tc {

using bf16 = __nv_bfloat16;

constexpr int TM = 128;          // cells per CTA (GEMM M)
constexpr int THREADS = 128;     // four warps: one TMEM lane quadrant each
constexpr int CORE = 128;        // bytes of one core matrix (8 rows x 16 B)
constexpr unsigned WAIT_LIMIT = 1u << 24;  // polls of an mbarrier before giving up

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

// Wait for the phase with the given parity to complete; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity) {
    const uint32_t a = smem_u32(bar);
    for (unsigned it = 0; it < WAIT_LIMIT; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n"
            " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after_sync() {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before_sync() {
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}

// Allocate `ncols` TMEM columns (one warp); the address is written to *dst (smem).
__device__ __forceinline__ void tmem_alloc(uint32_t *dst, unsigned ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(dst)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, unsigned ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols)
                 : "memory");
}

// Shared-memory matrix descriptor: start, leading- and stride-dimension byte
// offsets (all >> 4), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3fff);
    d |= (uint64_t)((lbo >> 4) & 0x3fff) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3fff) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::f16: bfloat16 A and B (both K-major),
// binary32 D, shape M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
    return (1u << 4)                       // D: binary32
           | (1u << 7)                     // A: bfloat16
           | (1u << 10)                    // B: bfloat16
           | ((uint32_t)(n >> 3) << 17)    // N / 8
           | ((uint32_t)(m >> 4) << 24);   // M / 16
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n"
        " setp.ne.u32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive on `bar` once all previously issued MMAs of this thread have completed.
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
            smem_u32(bar))
        : "memory");
}

// 32 lanes x 32 columns of binary32 from TMEM: thread t of the warp gets lane
// (warp's quadrant base + t), columns col .. col + 31.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int c = 0; c < 32; ++c) v[c] = __uint_as_float(r[c]);
}

__device__ __forceinline__ void cp16(void *smem, const void *gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(smem)), "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

enum { EPI_RELU_BF16 = 0, EPI_LINEAR_F32 = 1 };

constexpr int APITCH = (TM + 8) * 16;  // bytes of one 8-channel plane of an A tile (130 rows used)

// Bytes of dynamic shared memory: layer weights and two A tiles.
__host__ __device__ constexpr size_t smem_bytes(int cin, int npad) {
    return (size_t)27 * cin * npad * 2 + 2 * (size_t)(cin / 8) * APITCH;
}

struct ConvTcArgs {
    const bf16 *x;        // [cells][CIN] channels-last input
    const bf16 *w;        // weights in the shared-memory image order (see prep)
    const float *bias;    // [COUT]
    void *y;              // [cells][COUT] bf16 (ReLU) or binary32 (linear)
    int nx, ny, nz;
    int tiles;            // ny * nz * ceil(nx / TM)
    unsigned *err;        // set non-zero if a bounded wait ran out
};

// Persistent: CTA b computes tiles b, b + gridDim.x, ...  A tile is 128 cells
// of one x-row.  The nine (dy, dz) source rows of a tile are staged one after
// another, each with a one-cell halo on both sides (130 cells); the three dx
// taps of a row read the same staged rows through descriptors whose start is
// shifted by 0, 1 or 2 cells (16 bytes each): in the no-swizzle K-major layout
// with 128-byte M-direction core-matrix stride the M rows of a plane are
// simply consecutive 16-byte rows.  Staged row groups are double-buffered
// across tiles, so the copy of the next group always overlaps the MMAs of the
// current one.
//
// Weight image: w[((((tap * KC + kc) * NG + ng) * 8 + r) * 8 + c] holds
// W[co = 8 ng + r][ci = 8 kc + c][tap], zero for co >= COUT or ci >= cin_real.
template <int CIN, int COUT, int EPI>
__global__ void __launch_bounds__(THREADS) conv_tc_kernel(const ConvTcArgs a) {
    constexpr int NPAD = COUT < 16 ? 16 : COUT;
    constexpr int KC = CIN / 8;     // core-matrix columns along K per tap
    constexpr int NG = NPAD / 8;    // core-matrix rows along N
    constexpr int A_BYTES = KC * APITCH;
    constexpr int W_BYTES = 27 * KC * NG * CORE;
    constexpr uint32_t IDESC = idesc_bf16(TM, NPAD);
    static_assert(CIN % 16 == 0 && COUT % 8 == 0 && COUT <= 32, "shape");
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t bar[2];
    __shared__ uint32_t tmem_base;
    unsigned char *Ws = smem;
    unsigned char *As = smem + W_BYTES;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int segs = (a.nx + TM - 1) / TM;
    const int mine = a.tiles > (int)blockIdx.x ? (a.tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int groups = 9 * mine;

    if (warp == 0) tmem_alloc(&tmem_base, 32);
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    for (int i = tid; i < W_BYTES / 16; i += THREADS)
        cp16(Ws + 16 * i, reinterpret_cast<const unsigned char *>(a.w) + 16 * i);

    // Stage source row group G (tile G / 9, dz dy = G % 9) into buffer G & 1.
    auto load_group = [&](int G) {
        const int tile = (int)blockIdx.x + (G / 9) * (int)gridDim.x;
        const int grp = G % 9;
        const int row = tile / segs, seg = tile - row * segs;
        const int y = row % a.ny, z = row / a.ny;
        const int dz = grp / 3 - 1, dy = grp % 3 - 1;
        int yy = (y + dy) % a.ny, zz = (z + dz) % a.nz;
        yy = yy < 0 ? yy + a.ny : yy;
        zz = zz < 0 ? zz + a.nz : zz;
        const long long rbase = ((long long)zz * a.ny + yy) * a.nx;
        unsigned char *dst = As + (G & 1) * A_BYTES;
        for (int i = tid; i < (TM + 2) * KC; i += THREADS) {
            const int c = i / KC, kc = i - c * KC;  // consecutive threads: one cell's chunks
            int xx = (seg * TM - 1 + c) % a.nx;
            xx = xx < 0 ? xx + a.nx : xx;
            cp16(dst + kc * APITCH + c * 16, a.x + (rbase + xx) * CIN + 8 * kc);
        }
    };

    if (groups > 0) load_group(0);
    cp_commit();
    __syncthreads();  // barriers initialised, TMEM address published
    tc_fence_after_sync();
    const uint32_t tmem = tmem_base;
    bool abort = false;
    for (int G = 0; G < groups; ++G) {
        if (G + 1 < groups) {
            if (G >= 1) {  // the MMAs of group G-1 read the buffer group G+1 goes to
                const bool ok = mbar_wait(&bar[(G - 1) & 1], ((G - 1) >> 1) & 1);
                if (__syncthreads_or(!ok)) {
                    abort = true;
                    break;
                }
            }
            load_group(G + 1);
        }
        cp_commit();
        cp_wait<1>();          // group G (and the weights) have landed for this thread
        fence_proxy_async_smem();
        __syncthreads();       // ... for every thread; the last epilogue's TMEM reads are done
        const int grp = G % 9;
        if (tid == 0) {
            tc_fence_after_sync();
            const uint32_t abase = smem_u32(As + (G & 1) * A_BYTES);
            const uint32_t wbase = smem_u32(Ws);
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int kk = 0; kk < CIN / 16; ++kk) {
                    const int tap = grp * 3 + j;
                    const uint64_t ad = smem_desc(abase + j * 16 + kk * 2 * APITCH, APITCH, CORE);
                    const uint64_t bd =
                        smem_desc(wbase + ((tap * KC + 2 * kk) * NG) * CORE, NG * CORE, CORE);
                    mma_bf16(tmem, ad, bd, IDESC, (grp > 0 || j > 0 || kk > 0) ? 1u : 0u);
                }
            mma_commit(&bar[G & 1]);
        }
        if (grp == 8) {  // tile complete: epilogue
            const bool ok = mbar_wait(&bar[G & 1], (G >> 1) & 1);
            if (__syncthreads_or(!ok)) {
                abort = true;
                break;
            }
            tc_fence_after_sync();
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16), v);
            tc_fence_before_sync();
            const int tile = (int)blockIdx.x + (G / 9) * (int)gridDim.x;
            const int row = tile / segs, seg = tile - row * segs;
            const int y = row % a.ny, z = row / a.ny;
            const int x = seg * TM + warp * 32 + (tid & 31);
            if (x < a.nx) {
                const long long p = ((long long)z * a.ny + y) * a.nx + x;
                if (EPI == EPI_RELU_BF16) {
                    __align__(16) bf16 o[COUT];
#pragma unroll
                    for (int c = 0; c < COUT; ++c)
                        o[c] = __float2bfloat16_rn(fmaxf(v[c] + a.bias[c], 0.f));
                    uint4 *dst = reinterpret_cast<uint4 *>(static_cast<bf16 *>(a.y) + p * COUT);
#pragma unroll
                    for (int c = 0; c < COUT / 8; ++c) dst[c] = reinterpret_cast<const uint4 *>(o)[c];
                } else {
                    __align__(16) float o[COUT];
#pragma unroll
                    for (int c = 0; c < COUT; ++c) o[c] = v[c] + a.bias[c];
                    float4 *dst = reinterpret_cast<float4 *>(static_cast<float *>(a.y) + p * COUT);
#pragma unroll
                    for (int c = 0; c < COUT / 4; ++c) dst[c] = reinterpret_cast<const float4 *>(o)[c];
                }
            }
        }
    }
    cp_wait<0>();
    if (abort && tid == 0) atomicExch(a.err, 1u);
    tc_fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 32);
}

// Weight image for conv_tc_kernel from binary32 W[cout][cin_real][27].
__global__ void conv_tc_prep_kernel(const float *__restrict__ W, int cout, int cin_real, int cin,
                                    int npad, bf16 *__restrict__ img) {
    const int KC = cin / 8, NG = npad / 8;
    const int total = 27 * cin * npad;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int c = i & 7, r = (i >> 3) & 7;
        const int rest = i >> 6;  // (tap * KC + kc) * NG + ng
        const int ng = rest % NG;
        const int kc = (rest / NG) % KC;
        const int tap = rest / (NG * KC);
        const int co = 8 * ng + r, ci = 8 * kc + c;
        const float v = (co < cout && ci < cin_real) ? W[((long long)co * cin_real + ci) * 27 + tap] : 0.f;
        img[i] = __float2bfloat16_rn(v);
    }
}

}  // namespace tc
}  // namespace ac
