// Weight gradient of a 3x3x3 convolution (circular padding) on the tcgen05
// tensor cores:
//     dW[co][ci][kz][ky][kx] = sum_p dZ[co, p] X[ci, p + (kx - 1, ky - 1, kz - 1)],
// a GEMM with K = cells.  Both operands come straight from row-planar
// activations (layout in conv_tc.cuh), in which a cell's eight channels are
// one 16-byte row: staged by the TMA, a plane of 136 cells is a column of
// MN-major core matrices (8 channels x 8 cells, 128 contiguous bytes), K
// advancing by 128 bytes per core matrix and the next 8 channels one plane
// (2176 bytes) further.  A shift of the input by one cell (the kx taps) is a
// 16-byte shift of the operand's start.
//
// For an output tile (128 cells of row (y, z)), the nine input rows (y + ky - 1,
// z + kz - 1) are three consecutive z-slices of three rows each, which a ring
// of slices keeps contiguous in shared memory (the first two slots are mirrored
// after the last, so any three consecutive slices form one run of planes at a
// uniform stride).  GEMM M = 128 rows = 16 consecutive planes of that run
// (input row, channel group) x 8 channels; N = the output channels of dZ (8
// padded to 16 by a zero plane, or 32).  With 32 input channels the 36 planes
// of the run are covered by blocks starting at planes 0, 16 and 20 (the last
// overlaps the second; each plane's sums are taken from one block); with 8 input
// channels one block covers the 9 planes (the other rows are discarded).  Each
// (kx, block) pair owns an accumulator in TMEM for the CTA's whole run, so the
// sum over all cells a CTA processes stays on chip; at the end the epilogue
// warps write per-CTA partial sums, which a second kernel adds in binary64 in
// a fixed order.
//
// dZ is read from a copy without the periodic halo cells (zero there and in the
// padding), so the cells of a ragged last K-step past nx contribute nothing.
// Warp roles as in the forward kernel: warp 4 (one thread) issues the TMA copies,
// warp 5 the MMAs, warps 0-3 zero the accumulators and read them at the end.
// Every wait is bounded; on timeout the role records an error word and stops.
#pragma once

#include "conv_tc.cuh"

namespace ac {
namespace tc {

struct WgradTcArgs {
    float *part;  // [grid][NACC][NB][128] per-CTA partial sums
    int nx, ny, nz;
    int zc;       // tiles per column segment
    unsigned *err;
};

// Shape constants of the weight-gradient kernel for CIN input and COUT output channels.
template <int CIN, int COUT>
struct WgradShape {
    static constexpr int KC = CIN / 8;                       // planes per input row
    static constexpr int NPL = 9 * KC;                       // planes of the nine-row run
    static constexpr int NMB = NPL <= 16 ? 1 : (NPL + 15) / 16;  // M blocks per kx
    static constexpr int DKC = COUT < 16 ? 2 : COUT / 8;     // planes of a dZ tile
    static constexpr int NB = 8 * DKC;                       // GEMM N
    static constexpr int NACC = 3 * NMB;                     // accumulators (kx, block)
    static constexpr int TCOLS = NACC * NB <= 32 ? 32 : NACC * NB <= 64 ? 64 : NACC * NB <= 128 ? 128
                                 : NACC * NB <= 256 ? 256 : 512;
    static constexpr int NSLOT = KC == 1 ? 8 : 4;            // slice ring (plus two mirrors)
    static constexpr int ROW = KC * PLANE;
    static constexpr int SLICE = 3 * ROW;
    static constexpr int NDZ = 3;                            // dZ tile ring
    static constexpr int DZT = DKC * PLANE;
    // the last block of a run starts at plane NPL - 16 (0 for a single block)
    static constexpr int P0LAST = NMB == 1 ? 0 : NPL - 16;
    // bytes the A operand can reach from the last ring slot, or the mirrored ring
    static constexpr int RING_A = (NSLOT - 1) * SLICE + (P0LAST + 16) * PLANE;
    static constexpr int RING = RING_A > (NSLOT + 2) * SLICE ? RING_A : (NSLOT + 2) * SLICE;
    static constexpr size_t SMEM = (size_t)RING + (size_t)NDZ * DZT;
    static_assert(NACC * NB <= 512 && (CIN == 8 || CIN == 32) && (COUT == 8 || COUT == 32), "shape");
};

__host__ __device__ constexpr int wgrad_p0(int mb, int nmb, int npl) {
    return nmb == 1 ? 0 : (mb < nmb - 1 ? 16 * mb : npl - 16);
}

// Instruction descriptor with both operands MN-major (bits 15 and 16).
__host__ __device__ constexpr uint32_t idesc_bf16_mn(int m, int n) {
    return idesc_bf16(m, n) | (1u << 15) | (1u << 16);
}

template <int CIN, int COUT>
__global__ void __launch_bounds__(THREADS, 1)
    wgrad_tc_kernel(const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap dmap,
                    const WgradTcArgs a) {
    using S = WgradShape<CIN, COUT>;
    constexpr int KC = S::KC, NMB = S::NMB, NB = S::NB, NACC = S::NACC, NSLOT = S::NSLOT;
    constexpr int ROW = S::ROW, SLICE = S::SLICE, NDZ = S::NDZ, DZT = S::DZT;
    constexpr uint32_t SLICE_TX = 3 * KC * PLANE;
    constexpr uint32_t DZ_TX = S::DKC * PLANE;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t full[NSLOT], empty[NSLOT], dfull[NDZ], dempty[NDZ], done;
    __shared__ uint32_t tmem_base;
    unsigned char *Ss = smem;
    unsigned char *Ds = smem + S::RING;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int segs = (a.nx + TM - 1) / TM;
    const long long nseg = (long long)((a.nz + a.zc - 1) / a.zc) * a.ny * segs;
    ConvTcArgs ga;  // the fields segment_of reads
    ga.nx = a.nx;
    ga.ny = a.ny;
    ga.nz = a.nz;
    ga.zc = a.zc;

    if (warp == 0) tmem_alloc(&tmem_base, S::TCOLS);
    if (threadIdx.x == 128) {
        for (int b = 0; b < NSLOT; ++b) {
            mbar_init(&full[b], 1);
            mbar_init(&empty[b], 1);
        }
        for (int b = 0; b < NDZ; ++b) {
            mbar_init(&dfull[b], 1);
            mbar_init(&dempty[b], 1);
        }
        mbar_init(&done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    // the ring bytes past the mirrored slots are only read into discarded rows:
    // keep them finite
    for (int i = (NSLOT + 2) * SLICE + 16 * (int)threadIdx.x; i < S::RING; i += 16 * THREADS)
        *reinterpret_cast<uint4 *>(Ss + i) = make_uint4(0, 0, 0, 0);
    fence_proxy_async_smem();
    __syncthreads();  // barriers initialised, TMEM address published
    tc_fence_after_sync();
    const uint32_t tmem = tmem_base;
    if (warp < 4) {
        for (int k = 0; k < NACC; ++k) tmem_zero<NB>(tmem + ((uint32_t)(warp * 32) << 16) + k * NB);
        tc_fence_before_sync();
    }
    __syncthreads();
    tc_fence_after_sync();

    if (warp == 4) {
        if (lane == 0) {  // ---- TMA producer: slices 0, 1, then (slice i + 2, dZ tile i)
            long long s = 0, t = 0;
            bool ok = true;
            auto slice = [&](const Segment &sg, int j) {
                const int b = (int)(s % NSLOT);
                const long long k = s / NSLOT;
                if (k > 0 && !mbar_wait(&empty[b], (unsigned)((k - 1) & 1))) return false;
                const int copies = b < 2 ? 2 : 1;
                mbar_expect_tx(&full[b], copies * SLICE_TX);
                const int z = wrapi(sg.z0 + j - 1, a.nz);
                for (int c = 0; c < copies; ++c) {
                    unsigned char *dst = Ss + (b + c * NSLOT) * SLICE;
#pragma unroll
                    for (int r = 0; r < 3; ++r)
                        tma_load_5d(dst + r * ROW, &xmap, &full[b], 0, sg.seg * (TM / 8), 0,
                                    wrapi(sg.y + r - 1, a.ny), z);
                }
                ++s;
                return true;
            };
            for (long long g = blockIdx.x; g < nseg && ok; g += gridDim.x) {
                const Segment sg = segment_of(g, ga, segs);
                ok = slice(sg, 0) && slice(sg, 1);
                for (int i = 0; i < sg.len && ok; ++i) {
                    ok = slice(sg, i + 2);
                    if (!ok) break;
                    const int d = (int)(t % NDZ);
                    const long long k = t / NDZ;
                    if (k > 0 && !mbar_wait(&dempty[d], (unsigned)((k - 1) & 1))) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(&dfull[d], DZ_TX);
                    tma_load_5d(Ds + d * DZT, &dmap, &dfull[d], 0, sg.seg * (TM / 8), 0, sg.y,
                                sg.z0 + i);
                    ++t;
                }
            }
            if (!ok) atomicExch(a.err, 1u);
            // no copy may be in flight when the CTA exits: wait for each buffer's last fill
            for (int b = 0; b < NSLOT; ++b)
                if (s > b) mbar_wait(&full[b], (unsigned)(((s - 1 - b) / NSLOT) & 1));
            for (int d = 0; d < NDZ; ++d)
                if (t > d) mbar_wait(&dfull[d], (unsigned)(((t - 1 - d) / NDZ) & 1));
        }
    } else if (warp == 5) {
        // ---- MMA issuer: the whole warp runs the loop, one elected lane issues
        long long s = 0, t = 0;  // first slice of the current tile's run; dZ tiles consumed
        bool ok = true;
        const uint32_t idesc = idesc_bf16_mn(TM, NB);
        for (long long g = blockIdx.x; g < nseg && ok; g += gridDim.x) {
            const Segment sg = segment_of(g, ga, segs);
            const int L = sg.len;
            const int valid = a.nx - sg.seg * TM;
            const int nks = valid >= TM ? TM / 16 : (valid + 15) / 16;  // K-steps with cells < nx
            for (int i = 0; i < L; ++i) {
                // slices s .. s + 2 and dZ tile t have landed (the first two were
                // waited for by the previous tile of the segment, or are waited now)
                for (int q = (i == 0 ? 0 : 2); q < 3 && ok; ++q)
                    ok = __all_sync(0xffffffffu,
                                    mbar_wait(&full[(s + q) % NSLOT], (unsigned)(((s + q) / NSLOT) & 1)));
                const int d = (int)(t % NDZ);
                if (ok)
                    ok = __all_sync(0xffffffffu, mbar_wait(&dfull[d], (unsigned)((t / NDZ) & 1)));
                if (!ok) break;
                tc_fence_after_sync();
                const uint32_t abase = smem_u32(Ss + (int)(s % NSLOT) * SLICE);
                const uint32_t bbase = smem_u32(Ds + d * DZT) + 16;  // smem row k + 1 = cell x0 + k
                const uint64_t a0 = smem_desc(abase, CORE, PLANE);
                const uint64_t b0 = smem_desc(bbase, CORE, PLANE);
                for (int ks = 0; ks < nks; ++ks) {
#pragma unroll
                    for (int kx = 0; kx < 3; ++kx)
#pragma unroll
                        for (int mb = 0; mb < NMB; ++mb) {
                            const uint32_t aoff =
                                (uint32_t)(wgrad_p0(mb, NMB, S::NPL) * PLANE + (ks * 16 + kx) * 16);
                            const uint64_t ad = a0 + (aoff >> 4);
                            const uint64_t bd = b0 + ((uint32_t)(ks * 256) >> 4);
                            mma_bf16_elect(tmem + (uint32_t)((kx * NMB + mb) * NB), ad, bd, idesc);
                        }
                }
                mma_commit_elect(&dempty[d]);
                mma_commit_elect(&empty[s % NSLOT]);  // slice s serves no later tile
                if (i == L - 1) {
                    mma_commit_elect(&empty[(s + 1) % NSLOT]);
                    mma_commit_elect(&empty[(s + 2) % NSLOT]);
                    s += 3;
                } else {
                    s += 1;
                }
                ++t;
            }
        }
        if (!ok && lane == 0) atomicExch(a.err, 1u);
        mma_commit_elect(&done);  // every MMA of the CTA, before the epilogue reads TMEM
    } else {  // ---- epilogue: warps 0-3, TMEM lanes 32 warp .. 32 warp + 31
        const bool ok = __all_sync(0xffffffffu, mbar_wait(&done, 0));
        tc_fence_after_sync();
        if (ok) {
            const int m = warp * 32 + lane;
#pragma unroll 1
            for (int k = 0; k < NACC; ++k) {
                const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(k * NB);
                float v[NB];
                if constexpr (NB == 32)
                    tmem_ld32(taddr, v);
                else
                    tmem_ld16(taddr, v);
                float *dst = a.part + ((long long)blockIdx.x * NACC + k) * NB * TM + m;
#pragma unroll
                for (int n = 0; n < NB; ++n) dst[n * TM] = v[n];
            }
        } else if (lane == 0) {
            atomicExch(a.err, 1u);
        }
    }
    tc_fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, S::TCOLS);
}

// gW[co][ci][kz][ky][kx] (ci < cin_real) from the per-CTA partials: one thread
// per partial entry (accumulator k = kx * NMB + block, column co, row m), rows
// fastest so that the CTAs' blocks are read coalesced; entries that hold no
// gradient (padded columns and rows, planes another block owns) are skipped.
// Row m of block mb is plane P = P0(mb) + m / 8, channel 8 (P % KC) + m % 8,
// tap row P / KC = 3 kz + ky.  Binary64 sums in CTA order.
template <int CIN, int COUT>
__global__ void wgrad_tc_reduce_kernel(const float *__restrict__ part, int ctas, int cin_real,
                                       float *__restrict__ gW) {
    using S = WgradShape<CIN, COUT>;
    constexpr int PER_CTA = S::NACC * S::NB * TM;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < PER_CTA; t += gridDim.x * blockDim.x) {
        const int m = t % TM, co = (t / TM) % S::NB, k = t / (TM * S::NB);
        const int kx = k / S::NMB, mb = k % S::NMB;
        const int P = wgrad_p0(mb, S::NMB, S::NPL) + m / 8;
        if (co >= COUT || P >= S::NPL) continue;
        const int owner = S::NMB == 1 ? 0 : (P < 16 * (S::NMB - 1) ? P / 16 : S::NMB - 1);
        const int ci = 8 * (P % S::KC) + m % 8;
        if (owner != mb || ci >= cin_real) continue;
        const int tr = P / S::KC;
        double s = 0.0;
        for (int b = 0; b < ctas; ++b) s += part[(long long)b * PER_CTA + t];
        gW[(co * cin_real + ci) * 27 + tr * 3 + kx] = (float)s;
    }
}

}  // namespace tc
}  // namespace ac
