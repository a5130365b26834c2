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
// The sum is split by the input cell q (each tile's 128 cells):
//     dW_kx[ci][co] = sum_q X[ci, q] dZ[co, q + 1 - kx]   (for each (kz, ky) input row),
// so the A operand (the activations, rows of the tile's cells) is the same for
// the three kx taps and the B operand is dZ at three one-cell shifts.  The nine
// input rows (y + ky - 1, z + kz - 1) of a tile lie in three consecutive z-slices
// of three rows each, held in a ring of slices.  GEMM M = 128 rows = 16
// consecutive planes (input row, channel group) x 8 channels: with 32 input
// channels one block per slice (its 12 planes; the 4 planes after it are read
// into discarded rows), with 8 one block over the 9 planes of the three slices,
// kept contiguous by mirroring the ring's first two slots after its last.
// N = (kx, output channel): the TMA lands dZ's tile (with its periodic halo
// cells) beside three copy areas, and the epilogue warps, idle until the end,
// write the copies shifted by 0, 1 and 2 cells, plane after plane, so that one
// descriptor spans all three at a uniform stride (N = 3 x 16 or 3 x 32); rows of
// cells past nx (a ragged tile) are written as zeros, so those cells add nothing.
// Each M block owns an accumulator in TMEM for the CTA's
// whole run, so the sum over all cells a CTA processes stays on chip; at the end
// the epilogue warps write per-CTA partial sums, which a second kernel adds in
// binary64 in a fixed order.
//
// Warp roles: warp 4 (one thread) issues the TMA copies, warp 5 the MMAs, warps
// 0-3 zero the accumulators, prepare each dZ tile's shifted copies and read the
// accumulators at the end.  Every wait is bounded; on timeout the role records
// an error word and stops.
#pragma once

#include "conv_tc.cuh"

namespace ac {
namespace tc {

struct WgradTcArgs {
    float *part;  // [grid][NACC][N3][128] per-CTA partial sums
    int nx, ny, nz;
    int zc;       // tiles per column segment
    unsigned *err;
};

// Shape constants of the weight-gradient kernel for CIN input and COUT output channels.
template <int CIN, int COUT>
struct WgradShape {
    static constexpr int KC = CIN / 8;                       // planes per input row
    static constexpr int NPL = 9 * KC;                       // planes of the nine-row run
    // 32 input channels: one M block per slice (its 12 planes, 4 more rows discarded),
    // so no block crosses a slice and the ring needs no mirror; 8 input channels: one
    // block over the 9 planes of three slices kept contiguous by a mirrored ring
    static constexpr bool MIRROR = KC == 1;
    static constexpr int NMB = MIRROR ? 1 : 3;               // M blocks
    static constexpr int BLK = MIRROR ? 0 : 3 * KC;          // planes per block (stride of P0)
    static constexpr int DKC = COUT < 16 ? 2 : COUT / 8;     // planes of a dZ tile
    static constexpr int NB = 8 * DKC;                       // output channels (padded)
    static constexpr int N3 = 3 * NB;                        // GEMM N = (kx, channel)
    static constexpr int NACC = NMB;                         // accumulators (one per M block)
    static constexpr int TCOLS = NACC * N3 <= 32 ? 32 : NACC * N3 <= 64 ? 64 : NACC * N3 <= 128 ? 128
                                 : NACC * N3 <= 256 ? 256 : 512;
    static constexpr int NSLOT = MIRROR ? 8 : 5;             // slice ring (plus two mirrors)
    static constexpr int ROW = KC * PLANE;
    static constexpr int SLICE = 3 * ROW;
    static constexpr int NL = 2;                             // landed dZ tiles (TMA ring)
    static constexpr int NC = 2;                             // sets of three shifted copies
    static constexpr int COPY = DKC * PLANE;                 // one dZ tile (one copy)
    // bytes the A operand can reach past the start of the last ring slot: 16 planes
    // from its block's start (the mirrored ring: all blocks start in the first slot)
    static constexpr int RING_A = (NSLOT - 1) * SLICE + 16 * PLANE;
    static constexpr int RING_S = (MIRROR ? NSLOT + 2 : NSLOT) * SLICE;
    static constexpr int RING = RING_A > RING_S ? RING_A : RING_S;
    static constexpr size_t SMEM = (size_t)RING + (size_t)(3 * NC + NL) * COPY;
    static_assert(NACC * N3 <= 512 && N3 % 16 == 0 && N3 <= 256 && (CIN == 8 || CIN == 32) &&
                      (COUT == 8 || COUT == 32), "shape");
};



// Instruction descriptor with both operands MN-major (bits 15 and 16).
__host__ __device__ constexpr uint32_t idesc_bf16_mn(int m, int n) {
    return idesc_bf16(m, n) | (1u << 15) | (1u << 16);
}

template <int CIN, int COUT>
__global__ void __launch_bounds__(THREADS, 1)
    wgrad_tc_kernel(const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap dmap,
                    const WgradTcArgs a) {
    using S = WgradShape<CIN, COUT>;
    constexpr int KC = S::KC, NMB = S::NMB, N3 = S::N3, NACC = S::NACC, NSLOT = S::NSLOT;
    constexpr int ROW = S::ROW, SLICE = S::SLICE, NL = S::NL, NC = S::NC, DKC = S::DKC;
    constexpr int COPY = S::COPY;
    constexpr uint32_t SLICE_TX = 3 * KC * PLANE;
    constexpr uint32_t DZ_TX = DKC * PLANE;
    extern __shared__ __align__(1024) unsigned char smem[];
    // lfull: a dZ tile landed; lempty: its copies are taken; cready: a copy set is
    // written; cempty: the MMAs reading a copy set are done
    __shared__ uint64_t full[NSLOT], empty[NSLOT], lfull[NL], lempty[NL], cready[NC], cempty[NC], done;
    __shared__ uint32_t tmem_base;
    unsigned char *Ss = smem;
    unsigned char *Cs = smem + S::RING;             // copy sets, 3 COPY each
    unsigned char *Ls = Cs + 3 * NC * COPY;         // landed tiles
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
        for (int b = 0; b < NL; ++b) {
            mbar_init(&lfull[b], 1);
            mbar_init(&lempty[b], 4);
        }
        for (int b = 0; b < NC; ++b) {
            mbar_init(&cready[b], 4);
            mbar_init(&cempty[b], 1);
        }
        mbar_init(&done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    // the ring bytes past the slots are only read into discarded rows: keep them finite
    for (int i = S::RING_S + 16 * (int)threadIdx.x; i < S::RING; i += 16 * THREADS)
        *reinterpret_cast<uint4 *>(Ss + i) = make_uint4(0, 0, 0, 0);
    fence_proxy_async_smem();
    __syncthreads();  // barriers initialised, TMEM address published
    tc_fence_after_sync();
    const uint32_t tmem = tmem_base;
    if (warp < 4) {
        for (int k = 0; k < NACC * N3 / 16; ++k)
            tmem_zero<16>(tmem + ((uint32_t)(warp * 32) << 16) + k * 16);
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
                const int copies = S::MIRROR && b < 2 ? 2 : 1;
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
                    const int l = (int)(t % NL);
                    const long long k = t / NL;
                    if (k > 0 && !mbar_wait(&lempty[l], (unsigned)((k - 1) & 1))) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(&lfull[l], DZ_TX);
                    // landed row r = slot x0 + r, cell x0 + r - 1
                    tma_load_5d(Ls + l * COPY, &dmap, &lfull[l], 0, sg.seg * (TM / 8), 0, sg.y,
                                sg.z0 + i);
                    ++t;
                }
            }
            if (!ok) atomicExch(a.err, 1u);
            // no copy may be in flight when the CTA exits: wait for each buffer's last fill
            for (int b = 0; b < NSLOT; ++b)
                if (s > b) mbar_wait(&full[b], (unsigned)(((s - 1 - b) / NSLOT) & 1));
            for (int l = 0; l < NL; ++l)
                if (t > l) mbar_wait(&lfull[l], (unsigned)(((t - 1 - l) / NL) & 1));
        }
    } else if (warp == 5) {
        // ---- MMA issuer: the whole warp runs the loop, one elected lane issues
        long long s = 0, t = 0;  // first slice of the current tile's run; dZ tiles consumed
        bool ok = true;
        const uint32_t idesc = idesc_bf16_mn(TM, N3);
        for (long long g = blockIdx.x; g < nseg && ok; g += gridDim.x) {
            const Segment sg = segment_of(g, ga, segs);
            const int L = sg.len;
            const int valid = a.nx - sg.seg * TM;
            const int nks = valid >= TM ? TM / 16 : (valid + 15) / 16;  // K-steps with cells < nx
            for (int i = 0; i < L; ++i) {
                // slices s .. s + 2 have landed (the first two were waited for by the
                // previous tile of the segment, or are waited now); tile t's copies are ready
                for (int q = (i == 0 ? 0 : 2); q < 3 && ok; ++q)
                    ok = __all_sync(0xffffffffu,
                                    mbar_wait(&full[(s + q) % NSLOT], (unsigned)(((s + q) / NSLOT) & 1)));
                const int c = (int)(t % NC);
                if (ok)
                    ok = __all_sync(0xffffffffu, mbar_wait(&cready[c], (unsigned)((t / NC) & 1)));
                if (!ok) break;
                tc_fence_after_sync();
                // A: the tile's cells x0 + k are staged rows k + 1 of every plane of the run;
                // block mb starts at plane 0 of the run's (mb)-th slice
                uint64_t a0[NMB];
#pragma unroll
                for (int mb = 0; mb < NMB; ++mb)  // block mb: slice s + mb, in its own slot
                    a0[mb] = smem_desc(smem_u32(Ss + (int)((s + mb) % NSLOT) * SLICE) + 16, CORE, PLANE);
                const uint64_t b0 = smem_desc(smem_u32(Cs + c * 3 * COPY), CORE, PLANE);
                for (int ks = 0; ks < nks; ++ks) {
                    const uint64_t step = (uint32_t)(ks * 256) >> 4;
#pragma unroll
                    for (int mb = 0; mb < NMB; ++mb)
                        mma_bf16_elect(tmem + (uint32_t)(mb * N3), a0[mb] + step, b0 + step, idesc);
                }
                mma_commit_elect(&cempty[c]);
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
    } else {  // ---- warps 0-3: the dZ tiles' shifted copies, then TMEM lanes 32 warp ..
        const int tid = threadIdx.x;  // 0 .. 127
        bool ok = true;
        long long t = 0;
        for (long long g = blockIdx.x; g < nseg && ok; g += gridDim.x) {
            const Segment sg = segment_of(g, ga, segs);
            const int valid = a.nx - sg.seg * TM;  // rows r < valid are cells < nx
            for (int i = 0; i < sg.len; ++i, ++t) {
                const int l = (int)(t % NL), c = (int)(t % NC);
                ok = __all_sync(0xffffffffu, mbar_wait(&lfull[l], (unsigned)((t / NL) & 1)));
                if (ok && t >= NC)  // the MMAs of tile t - NC have read this copy set
                    ok = __all_sync(0xffffffffu,
                                    mbar_wait(&cempty[c], (unsigned)(((t / NC) - 1) & 1)));
                if (!ok) break;
                unsigned char *base = Cs + c * 3 * COPY;  // copy kx at base + kx * COPY
                const unsigned char *landed = Ls + l * COPY;
                // copy kx, row r = landed row r + 2 - kx (cell x0 + r + 1 - kx); rows of
                // cells past nx (r >= valid) zero
                for (int e = tid; e < DKC * TM; e += 128) {
                    const int pl = e / TM, r = e - pl * TM;
                    const uint4 *src = reinterpret_cast<const uint4 *>(landed + pl * PLANE);
                    const uint4 z = make_uint4(0, 0, 0, 0);
                    const bool in = r < valid;
                    reinterpret_cast<uint4 *>(base + 2 * COPY + pl * PLANE)[r] = in ? src[r] : z;
                    reinterpret_cast<uint4 *>(base + COPY + pl * PLANE)[r] = in ? src[r + 1] : z;
                    reinterpret_cast<uint4 *>(base + pl * PLANE)[r] = in ? src[r + 2] : z;
                }
                // generic reads of the landed tile before the TMA refills it, generic
                // writes of the copies before the tensor core reads them
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(&lempty[l]);
                    mbar_arrive(&cready[c]);
                }
            }
        }
        if (ok) ok = __all_sync(0xffffffffu, mbar_wait(&done, 0));
        tc_fence_after_sync();
        if (ok) {
            const int m = warp * 32 + lane;
            constexpr int CH = N3 % 32 == 0 ? 32 : 16;
#pragma unroll 1
            for (int k = 0; k < NACC; ++k)
#pragma unroll 1
                for (int c0 = 0; c0 < N3; c0 += CH) {
                    const uint32_t taddr =
                        tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(k * N3 + c0);
                    float v[CH];
                    if constexpr (CH == 32)
                        tmem_ld32(taddr, v);
                    else
                        tmem_ld16(taddr, v);
                    float *dst = a.part + (((long long)blockIdx.x * NACC + k) * N3 + c0) * TM + m;
#pragma unroll
                    for (int n = 0; n < CH; ++n) dst[n * TM] = v[n];
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
// per partial entry (M block mb, column n = kx NB + co, row m), rows fastest so
// that the CTAs' blocks are read coalesced; entries that hold no gradient (padded
// columns, rows past a block's planes) are skipped.  Row m of block mb is plane
// P = mb BLK + m / 8 of the run, channel 8 (P % KC) + m % 8, tap row P / KC = 3 kz + ky.
// Binary64 sums in CTA order.
template <int CIN, int COUT>
__global__ void wgrad_tc_reduce_kernel(const float *__restrict__ part, int ctas, int cin_real,
                                       float *__restrict__ gW) {
    using S = WgradShape<CIN, COUT>;
    constexpr int PER_CTA = S::NACC * S::N3 * TM;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < PER_CTA; t += gridDim.x * blockDim.x) {
        const int m = t % TM, n = (t / TM) % S::N3, mb = t / (TM * S::N3);
        const int kx = n / S::NB, co = n % S::NB;
        const int P = mb * S::BLK + m / 8;
        if (co >= COUT || P >= S::NPL || (S::BLK > 0 && m / 8 >= S::BLK)) continue;
        const int ci = 8 * (P % S::KC) + m % 8;
        if (ci >= cin_real) continue;
        const int tr = P / S::KC;
        double s = 0.0;
        for (int b = 0; b < ctas; ++b) s += part[(long long)b * PER_CTA + t];
        gW[(co * cin_real + ci) * 27 + tr * 3 + kx] = (float)s;
    }
}

}  // namespace tc
}  // namespace ac
