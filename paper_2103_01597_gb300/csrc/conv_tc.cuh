// 3-D convolution (3x3x3 taps, circular padding) as an implicit GEMM on the
// fifth-generation tensor cores: tcgen05.mma with bfloat16 operands from
// shared memory, staged by the tensor memory accelerator (TMA), and binary32
// accumulators in tensor memory (TMEM).
//
// Activation layout ("row-planar", RP): bfloat16, for each row (y, z) and each
// group kc of 8 channels a plane of nxp = roundup(nx + 2, 8) cells x 16 bytes,
// the first nx + 2 being x = nx-1, 0, 1, ..., nx-1, 0 (the periodic x halo is
// stored with the row; the rest is padding):
//     a[(((z * ny + y) * KC + kc) * nxp + x + 1) * 8 + c]  = channel 8 kc + c.
// The TMA sees a plane as rows of 128 bytes (8 cells x 8 channels), so every
// request is a whole line.  A box of 17 such rows x KC planes lands in shared
// memory as KC planes of 136 consecutive 16-byte cell rows, which is the
// canonical K-major no-swizzle operand layout (core matrices of 8 cells x 8
// channels) with M-direction core-matrix stride 128 bytes and K-direction
// stride 2176 bytes; the three dx taps of a row are the same operand started
// 0, 1 or 2 cells in (rows 130..135 are staged but never read).
//
// An output tile is 128 cells of one x-row (GEMM M = 128) for all output
// channels (N = COUT, padded to 16); K = 27 taps x CIN.  Warp roles in a
// persistent CTA: warp 4 (one thread) issues the TMA copies of z-slices
// (rows y-1, y, y+1 of one plane) into a six-slice ring; warp 5 (one thread)
// issues the MMAs of each tile into one of two TMEM accumulators and signals
// completion with tcgen05.commit; warps 0-3 read an accumulator back
// (tcgen05.ld, one TMEM lane per thread), add the bias, apply ReLU and store.
// A CTA marches along z through column segments, so each staged slice serves
// three tiles.  Every wait is bounded: on timeout a role records an error
// word and stops, the others run out of their own bounded waits, and TMEM is
// still freed.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "bounds.cuh"

namespace ac {
namespace tc {

using bf16 = __nv_bfloat16;

constexpr int TM = 128;          // cells per tile (GEMM M)
constexpr int THREADS = 192;     // warps 0-3 epilogue (one TMEM lane quadrant each), 4 TMA, 5 MMA
constexpr int CORE = 128;        // bytes of one core matrix (8 rows x 16 B)
constexpr int PCELLS = TM + 8;          // cells of a staged plane (130 used)
constexpr int PLANE = PCELLS * 16;      // bytes of one staged 8-channel plane
constexpr int NBUF = 6;          // z-slices in the shared-memory ring
// Bounds of every wait, set by time: a try_wait poll of a phase that does not
// complete returns after about 3.8 us (measured on GB300), so 2^18 polls give
// up after about one second; a round of non-blocking tests takes well under a
// microsecond, so 2^23 rounds bound the issuer's waits to about a second too.
constexpr unsigned WAIT_LIMIT = 1u << 18;  // try_wait polls of an mbarrier before giving up
constexpr unsigned TEST_LIMIT = 1u << 23;  // rounds of non-blocking tests before giving up

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

// Wait for the phase with the given parity to complete, giving up after
// `limit` tests; false on timeout.
__device__ __forceinline__ bool mbar_wait_n(uint64_t *bar, unsigned parity, unsigned limit) {
    const uint32_t a = smem_u32(bar);
    for (unsigned it = 0; it < limit; ++it) {
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

__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity) {
    return mbar_wait_n(bar, parity, WAIT_LIMIT);
}

// A CTA that waits on a phase nothing completes, through the same bounded wait
// as the kernels above: err[0] = 1 once the wait has given up (the expected
// outcome), 0 if it completed.  Exercises the timeout path without a fault.
__global__ void wait_timeout_kernel(unsigned limit, unsigned *err) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) err[0] = mbar_wait_n(&bar, 0, limit) ? 0u : 1u;
}

// Six mbarrier phase tests issued back to back (their shared-memory latencies
// overlap); bit k of the result is set if phase (addr[k], par[k]) has completed.
__device__ __forceinline__ uint32_t mbar_test6(const uint32_t (&addr)[6], const unsigned (&par)[6]) {
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p0, p1, p2, p3, p4, p5;\n .reg .b32 t0, t1, t2, t3, t4, t5;\n"
        " mbarrier.test_wait.parity.shared::cta.b64 p0, [%1], %7;\n"
        " mbarrier.test_wait.parity.shared::cta.b64 p1, [%2], %8;\n"
        " mbarrier.test_wait.parity.shared::cta.b64 p2, [%3], %9;\n"
        " mbarrier.test_wait.parity.shared::cta.b64 p3, [%4], %10;\n"
        " mbarrier.test_wait.parity.shared::cta.b64 p4, [%5], %11;\n"
        " mbarrier.test_wait.parity.shared::cta.b64 p5, [%6], %12;\n"
        " selp.b32 t0, 1, 0, p0;\n selp.b32 t1, 2, 0, p1;\n selp.b32 t2, 4, 0, p2;\n"
        " selp.b32 t3, 8, 0, p3;\n selp.b32 t4, 16, 0, p4;\n selp.b32 t5, 32, 0, p5;\n"
        " or.b32 t0, t0, t1;\n or.b32 t2, t2, t3;\n or.b32 t4, t4, t5;\n"
        " or.b32 t0, t0, t2;\n or.b32 %0, t0, t4;\n}\n"
        : "=r"(r)
        : "r"(addr[0]), "r"(addr[1]), "r"(addr[2]), "r"(addr[3]), "r"(addr[4]), "r"(addr[5]),
          "r"(par[0]), "r"(par[1]), "r"(par[2]), "r"(par[3]), "r"(par[4]), "r"(par[5])
        : "memory");
    return r;
}

// Warp-wide wait for the phases whose bit is set in `pending` (every address
// must be a valid barrier; the others are tested and ignored).  Returns the
// same value on every lane: false if a lane gave up after TEST_LIMIT rounds.
__device__ __forceinline__ bool mbar_wait6_warp(const uint32_t (&addr)[6], const unsigned (&par)[6],
                                                uint32_t pending) {
    for (unsigned it = 0; it < TEST_LIMIT && pending; ++it) pending &= ~mbar_test6(addr, par);
    return __all_sync(0xffffffffu, pending == 0);
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

// A bfloat16 MMA (accumulating), issued by one elected lane of a converged warp.  The issuing loop runs
// on the whole warp so that its descriptors stay warp-uniform; with the loop
// inside a one-lane branch the MMA stream measured ~10% slower.
__device__ __forceinline__ void mma_bf16_elect(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                               uint32_t idesc) {
    asm volatile(
        "{\n .reg .pred p, e;\n .reg .b32 r;\n"
        " elect.sync r|e, 0xffffffff;\n"
        " setp.ne.u32 p, 1, 0;\n"
        " @e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc)
        : "memory");
}

// Arrive on `bar` once all MMAs issued so far by this warp have completed (one
// elected lane).
__device__ __forceinline__ void mma_commit_elect(uint64_t *bar) {
    asm volatile(
        "{\n .reg .pred e;\n .reg .b32 r;\n"
        " elect.sync r|e, 0xffffffff;\n"
        " @e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n}\n" ::"r"(
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

// 32 lanes x 16 columns of binary32 from TMEM.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int c = 0; c < 16; ++c) v[c] = __uint_as_float(r[c]);
}

// Zero 32 lanes x NB (16 or 32) columns of TMEM and wait for the stores.
template <int NB>
__device__ __forceinline__ void tmem_zero(uint32_t taddr) {
    const uint32_t z = 0;
    if (NB == 32)
        asm volatile(
            "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
            "{%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,"
            "%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};\n" ::"r"(taddr),
            "r"(z)
            : "memory");
    else
        asm volatile(
            "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
            "{%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};\n" ::"r"(taddr),
            "r"(z)
            : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// 5-D tiled TMA load of one box into shared memory, completing on `bar`.
__device__ __forceinline__ void tma_load_5d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0,
                                            int c1, int c2, int c3, int c4) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%3, %4, %5, %6, %7}], [%2];\n" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2),
        "r"(c3), "r"(c4)
        : "memory");
}

// Untiled bulk copy global -> shared (16-byte aligned, size a multiple of 16).
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Epilogues: ReLU to row-planar bfloat16 (hidden layers), or the network output
// scaled per channel to eight binary32 channel-major arrays (optionally with the
// largest |value|, NaN counting as largest, folded into a guard word), or (the
// input gradient through a ReLU, training) the value where the forward
// activation at the same cell and channel (row-planar `mask`) is positive, else
// 0, as row-planar bfloat16 (one-CTA kernel only).
enum { EPI_RELU_BF16 = 0, EPI_SCALED_F32 = 1, EPI_MASK_BF16 = 2 };

// Bytes of one staged row (KC planes, rounded up so rows stay 128-byte aligned).
__host__ __device__ constexpr int row_bytes(int cin) { return (cin / 8) * PLANE; }

// Padded row length (cells) of the row-planar layout.
__host__ __device__ constexpr int rp_cells(int nx) { return (nx + 2 + 7) / 8 * 8; }

// Bytes of the kz-stacked weight image (nb accumulator columns per tile): nine
// (ky, kx) taps x cin channels, or, for cin = 8, five tap pairs x 16 channels.
__host__ __device__ constexpr int w_bytes(int cin, int nb) {
    return cin == 8 ? 10 * 3 * nb * 16 : 9 * cin * 3 * nb * 2;
}

// Bytes of dynamic shared memory: the weight image and the slice ring.
__host__ __device__ constexpr size_t smem_bytes(int cin, int nb) {
    return (size_t)w_bytes(cin, nb) + (size_t)NBUF * 3 * row_bytes(cin);
}

// Layers with 8 input channels fill the K = 16 of an MMA with two taps of one
// slice: the pairs (tap a, tap b) below, tap = 3 dy + dx, the second core-matrix
// column of K lying (offset of b - offset of a) bytes after the first.  The last
// pair repeats tap 7 with zero weights.
__host__ __device__ constexpr int pair_tap(int p, int h) {
    return h == 0 ? (p < 4 ? 2 * p : 7) : (p < 4 ? 2 * p + 1 : 8);
}

// One 16-byte store of eight channels into a row-planar activation (element
// offset e); the checked build skips it if [e, e + 8) leaves the array.
#ifdef AC_BOUNDS_CHECK
__device__ __forceinline__ void store_rp(bf16 *Y, long long e, long long lim, uint4 v) {
    if (AC_BC_RANGE(e, 8, lim, AC_BC_CONV_ACT)) *reinterpret_cast<uint4 *>(Y + e) = v;
}
#else
__device__ __forceinline__ void store_rp(bf16 *Y, long long e, uint4 v) {
    *reinterpret_cast<uint4 *>(Y + e) = v;
}
#endif

struct ConvTcArgs {
    const bf16 *w;        // weights in the shared-memory image order (see prep)
    const float *bias;    // [COUT] (not read by EPI_MASK_BF16)
    bf16 *y;              // EPI_RELU_BF16, EPI_MASK_BF16: row-planar output (or null)
    const bf16 *mask;     // EPI_MASK_BF16: row-planar forward activation (COUT channels)
    float *out[8];        // EPI_SCALED_F32: channel c to out[c][cell]
    const float *out_scale;        // EPI_SCALED_F32: [8]
    unsigned long long *gmax;      // EPI_SCALED_F32: guard word (binary64 bits), or null
    int nx, ny, nz;
    int zc;               // tiles per column segment (z extent of a chunk)
    unsigned *err;        // set non-zero if a bounded wait ran out
};

__device__ __forceinline__ int wrapi(int v, int n) {
    if (v >= 0 && v < n) return v;
    const int m = v % n;
    return m < 0 ? m + n : m;
}

// Column segments: g = chunk * ncols + col (chunk-major, so that the CTAs of
// one wave work in the same z-chunk and share its slices in L2), col = y * segs
// + seg; a segment is the tiles z = chunk * zc ... of column col.
struct Segment {
    int y, seg, z0, len;
};

__device__ __forceinline__ Segment segment_of(long long g, const ConvTcArgs &a, int segs) {
    const long long ncols = (long long)a.ny * segs;
    const int chunk = (int)(g / ncols);
    const int col = (int)(g - chunk * ncols);
    Segment s;
    s.y = col / segs;
    s.seg = col - s.y * segs;
    s.z0 = chunk * a.zc;
    s.len = min(a.zc, a.nz - s.z0);
    return s;
}

// Persistent CTA g-loop over column segments b, b + G, ...  Slices are numbered
// in the order the CTA stages them (a segment of L tiles stages L + 2: planes
// z0-1 .. z0+L); slice s lives in ring buffer s % NBUF, as that buffer's
// (s / NBUF)-th fill.
//
// One MMA batch per slice.  Slice j of a segment (plane z0 + j - 1) feeds the
// tiles j-2, j-1, j of the segment that exist (dz = +1, 0, -1).  The weight
// image stacks the three kz blocks along N, [W(kz=2); W(kz=1); W(kz=0)], NB
// rows each, so the contributions of one slice to up to three tiles are one
// MMA of N = 3 NB (fewer at segment ends) whose accumulator is three
// consecutive NB-column blocks of TMEM: tile i of a segment owns block i, so
// the window of a slice never wraps (a segment has at most RBLK tiles).
// Because one MMA both opens a tile and adds to older ones, MMAs always
// accumulate, and blocks are zero when handed over: zeroed once at start and
// again by the epilogue after it reads a tile.  Barriers, each waited on in
// phase order:
//   full[b]  : TMA bytes of a fill landed (producer expect_tx, TMA complete_tx);
//   empty[b] : the MMAs reading a fill have finished (tcgen05.commit);
//   accf[k]  : the tile in block k is complete (commit after its third slice);
//   acce[k]  : the four epilogue warps have read and re-zeroed block k;
//   wbar     : the layer's weight image landed;
//   fin      : every MMA of the CTA has finished (before TMEM is freed).
//
// Weight image: w[(((kq * NGS + ng) * 8 + r) * 8 + c], NGS = 3 NB / 8, holds for
// stack row 8 ng + r = (2 - kz) NB + co the weight W[co][ci][kz][dyx] (dyx =
// 3 ky + kx) of K-chunk kq: kq = dyx * KC + kc and ci = 8 kc + c, or for
// CIN = 8, kq = 2 p + h, dyx = pair_tap(p, h) and ci = c; zero for co >= COUT,
// ci >= cin_real and the zero half of the last pair.
constexpr int RBLK = 16;  // TMEM accumulator blocks per CTA (>= tiles per segment, <= 32)
constexpr int GROUP = 3;  // slices the MMA issuer waits for at once (<= NBUF / 2)

template <int CIN, int COUT, int EPI>
__global__ void __launch_bounds__(THREADS, 1)
    conv_tc_kernel(const __grid_constant__ CUtensorMap xmap, const ConvTcArgs a) {
    constexpr int NB = COUT < 16 ? 16 : COUT;  // accumulator columns per tile
    constexpr int KC = CIN / 8;                // core-matrix columns along K per tap
    constexpr bool PAIR = CIN == 8;            // two taps per MMA
    constexpr int NGS = 3 * NB / 8;            // core-matrix rows of the kz stack
    constexpr int ROW = row_bytes(CIN);
    constexpr int SLICE = 3 * ROW;
    constexpr int W_BYTES = w_bytes(CIN, NB);
    constexpr uint32_t SLICE_TX = 3 * KC * PLANE;
    constexpr uint32_t TCOLS = RBLK * NB;      // 256 or 128 TMEM columns
    static_assert((CIN % 16 == 0 || CIN == 8) && COUT % 8 == 0 && COUT <= 32, "shape");
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t full[NBUF], empty[NBUF], accf[RBLK], acce[RBLK], wbar, fin;
    __shared__ uint32_t tmem_base;
    unsigned char *Ws = smem;
    unsigned char *Ss = smem + W_BYTES;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int segs = (a.nx + TM - 1) / TM;
    const long long nseg = (long long)((a.nz + a.zc - 1) / a.zc) * a.ny * segs;

    if (warp == 0) tmem_alloc(&tmem_base, TCOLS);
    if (threadIdx.x == 128) {
        for (int b = 0; b < NBUF; ++b) {
            mbar_init(&full[b], 1);
            mbar_init(&empty[b], 1);
        }
        for (int b = 0; b < RBLK; ++b) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], 4);
        }
        mbar_init(&wbar, 1);
        mbar_init(&fin, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();  // barriers initialised, TMEM address published
    tc_fence_after_sync();
    const uint32_t tmem = tmem_base;
    if (warp < 4) {  // every accumulator block starts at zero
        for (int k = 0; k < RBLK; ++k) tmem_zero<NB>(tmem + ((uint32_t)(warp * 32) << 16) + k * NB);
        tc_fence_before_sync();
    }
    __syncthreads();
    tc_fence_after_sync();

    if (warp == 4) {
        if (lane == 0) {  // ---- TMA producer
            mbar_expect_tx(&wbar, W_BYTES);
            bulk_load(Ws, a.w, W_BYTES, &wbar);
            long long s = 0;
            bool ok = true;
            for (long long g = blockIdx.x; g < nseg && ok; g += gridDim.x) {
                const Segment sg = segment_of(g, a, segs);
                for (int j = 0; j < sg.len + 2; ++j, ++s) {
                    const int b = (int)(s % NBUF);
                    const long long k = s / NBUF;
                    if (k > 0 && !mbar_wait(&empty[b], (unsigned)((k - 1) & 1))) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(&full[b], SLICE_TX);
                    const int z = wrapi(sg.z0 + j - 1, a.nz);
                    unsigned char *dst = Ss + b * SLICE;
#pragma unroll
                    for (int r = 0; r < 3; ++r)
                        tma_load_5d(dst + r * ROW, &xmap, &full[b], 0, sg.seg * (TM / 8), 0,
                                    wrapi(sg.y + r - 1, a.ny), z);
                }
            }
            if (!ok) atomicExch(a.err, 1u);
            // no copy may be in flight when the CTA exits: wait for each buffer's last fill
            mbar_wait(&wbar, 0);
            for (int b = 0; b < NBUF; ++b)
                if (s > b) mbar_wait(&full[b], (unsigned)(((s - 1 - b) / NBUF) & 1));
        }
    } else if (warp == 5) {
        {  // ---- MMA issuer: the whole warp runs the loop, one elected lane issues
            static_assert(GROUP == 3, "the combined wait tests six barriers");
            bool ok = __all_sync(0xffffffffu, mbar_wait(&wbar, 0));
            long long s = 0;  // slices consumed
            // per TMEM block: bit k of `used` = block k has held a tile, bit k of
            // `par` = parity of the number of tiles it has held (registers, not an
            // indexed array: local memory would sit on the issue path)
            uint32_t used = 0, par = 0;
            const uint32_t wbase = smem_u32(Ws);
            for (long long g = blockIdx.x; g < nseg && ok; g += gridDim.x) {
                const Segment sg = segment_of(g, a, segs);
                const int L = sg.len;
                for (int j = 0; j < L + 2; ++j, ++s) {
                    const int b = (int)(s % NBUF);
                    if (j % GROUP == 0) {
                        // one combined wait for the next GROUP slices: each landed,
                        // and each tile they open has been read out of its block
                        uint32_t addr[2 * GROUP];
                        unsigned want[2 * GROUP];
                        uint32_t pending = 0;
#pragma unroll
                        for (int q = 0; q < GROUP; ++q) {
                            const long long sq = s + q;
                            const int jq = j + q;
                            addr[2 * q] = smem_u32(&full[sq % NBUF]);
                            want[2 * q] = (unsigned)((sq / NBUF) & 1);
                            addr[2 * q + 1] = smem_u32(&acce[jq < RBLK ? jq : 0]);
                            want[2 * q + 1] = ((par >> jq) & 1u) ^ 1u;
                            if (jq < L + 2) pending |= 1u << (2 * q);
                            if (jq < L && ((used >> jq) & 1u)) pending |= 1u << (2 * q + 1);
                        }
                        ok = mbar_wait6_warp(addr, want, pending);
                        if (!ok) break;
                        tc_fence_after_sync();
                    }
                    if (j < L) {  // tile j opens in block j
                        used |= 1u << j;
                        par ^= 1u << j;
                    }
                    const int ta = j - 2 > 0 ? j - 2 : 0;
                    const int tb = j < L - 1 ? j : L - 1;
                    const uint32_t sbase = smem_u32(Ss + b * SLICE);
                    const uint32_t dtm = tmem + (uint32_t)(ta * NB);
                    const int stack0 = ta - j + 2;  // kz block of the first tile
                    const uint32_t idesc = idesc_bf16(TM, (tb - ta + 1) * NB);
                    // descriptors of the first operands; every other MMA adds a
                    // compile-time byte offset / 16 to the start-address field
                    const uint64_t b0 = smem_desc(wbase + stack0 * (NB / 8) * CORE, NGS * CORE, CORE);
                    if constexpr (PAIR) {
                        const uint64_t a0 = smem_desc(sbase, 0, CORE);
#pragma unroll
                        for (int p = 0; p < 5; ++p) {
                            const int ta0 = pair_tap(p, 0), tb0 = pair_tap(p, 1);
                            const uint32_t off = (ta0 / 3) * ROW + (ta0 % 3) * 16;
                            const uint32_t lbo = (tb0 / 3) * ROW + (tb0 % 3) * 16 - off;
                            const uint64_t ad = a0 + (off >> 4) + ((uint64_t)(lbo >> 4) << 16);
                            const uint64_t bd = b0 + ((2 * p * NGS * CORE) >> 4);
                            mma_bf16_elect(dtm, ad, bd, idesc);
                        }
                    } else {
                        const uint64_t a0 = smem_desc(sbase, PLANE, CORE);
#pragma unroll
                        for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                            for (int dx = 0; dx < 3; ++dx)
#pragma unroll
                                for (int kk = 0; kk < CIN / 16; ++kk) {
                                    const int dyx = dy * 3 + dx;
                                    const uint64_t ad = a0 + ((dy * ROW + dx * 16 + kk * 2 * PLANE) >> 4);
                                    const uint64_t bd = b0 + (((dyx * KC + 2 * kk) * NGS * CORE) >> 4);
                                    mma_bf16_elect(dtm, ad, bd, idesc);
                                }
                    }
                    mma_commit_elect(&empty[b]);
                    if (j >= 2) mma_commit_elect(&accf[j - 2]);  // tile j-2 has had its third slice
                }
            }
            if (!ok && lane == 0) atomicExch(a.err, 1u);
            // no MMA may be in flight when TMEM is freed: a final commit covers all
            mma_commit_elect(&fin);
            mbar_wait(&fin, 0);
        }
    } else {  // ---- epilogue: warps 0-3, TMEM lanes 32 warp .. 32 warp + 31
        float bias[COUT];
#pragma unroll
        for (int c = 0; c < COUT; ++c) bias[c] = EPI == EPI_MASK_BF16 ? 0.f : a.bias[c];
        float gm = 0.f;  // EPI_SCALED_F32: this thread's largest |output| (NaN if any)
        uint32_t par = 0;  // bit k: parity of the tiles block k has held so far
        bool ok = true;
        // EPI_MASK_BF16: the mask of the next tile is loaded while this one is
        // written (otherwise every tile would wait for a global round trip)
        constexpr int MK = EPI == EPI_MASK_BF16 ? COUT / 8 : 1;
        uint4 mnext[MK];
        auto load_mask = [&](int y, int x, int z, uint4(&m)[MK]) {
            if constexpr (EPI == EPI_MASK_BF16) {
                if (x >= a.nx) return;
                AC_BC_ONLY(const long long lim = (long long)rp_cells(a.nx) * a.ny * a.nz * COUT;)
#pragma unroll
                for (int kc = 0; kc < MK; ++kc) {
                    const long long e =
                        ((((long long)z * a.ny + y) * MK + kc) * rp_cells(a.nx) + x + 1) * 8;
                    m[kc] = *reinterpret_cast<const uint4 *>(a.mask + AC_BC(e, lim, AC_BC_CONV_ACT));
                }
            }
        };
        auto load_mask_seg = [&](long long g) {  // first tile of segment g
            if (g >= nseg) return;
            const Segment s2 = segment_of(g, a, segs);
            load_mask(s2.y, s2.seg * TM + warp * 32 + lane, s2.z0, mnext);
        };
        load_mask_seg(blockIdx.x);
        for (long long g = blockIdx.x; g < nseg && ok; g += gridDim.x) {
            const Segment sg = segment_of(g, a, segs);
            const int x = sg.seg * TM + warp * 32 + lane;
            for (int i = 0; i < sg.len; ++i) {
                const int kb = i;
                ok = __all_sync(0xffffffffu, mbar_wait(&accf[kb], (par >> kb) & 1u));
                par ^= 1u << kb;
                if (!ok) break;
                tc_fence_after_sync();
                const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(kb * NB);
                float v[NB];
                if constexpr (NB == 32)
                    tmem_ld32(taddr, v);
                else
                    tmem_ld16(taddr, v);
                tmem_zero<NB>(taddr);
                tc_fence_before_sync();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acce[kb]);
                uint4 mcur[MK];
#pragma unroll
                for (int kc = 0; kc < MK; ++kc) mcur[kc] = mnext[kc];
                if (EPI == EPI_MASK_BF16) {
                    if (i + 1 < sg.len)
                        load_mask(sg.y, x, sg.z0 + i + 1, mnext);
                    else
                        load_mask_seg(g + gridDim.x);
                }
                if (x >= a.nx) continue;
                const int z = sg.z0 + i;
                if (EPI == EPI_RELU_BF16 || EPI == EPI_MASK_BF16) {
                    __align__(16) bf16 o[COUT];
                    AC_BC_ONLY(const long long lim =
                                   (long long)rp_cells(a.nx) * a.ny * a.nz * COUT;)
#pragma unroll
                    for (int kc = 0; kc < COUT / 8; ++kc) {
                        const long long plane =
                            ((((long long)z * a.ny + sg.y) * (COUT / 8) + kc) * rp_cells(a.nx)) * 8;
                        if constexpr (EPI == EPI_MASK_BF16) {
                            __align__(16) bf16 m[8];
                            *reinterpret_cast<uint4 *>(m) = mcur[kc];
#pragma unroll
                            for (int c = 0; c < 8; ++c)
                                o[8 * kc + c] = __bfloat162float(m[c]) > 0.f
                                                    ? __float2bfloat16_rn(v[8 * kc + c])
                                                    : __float2bfloat16_rn(0.f);
                        } else {
#pragma unroll
                            for (int c = 0; c < 8; ++c)
                                o[8 * kc + c] =
                                    __float2bfloat16_rn(fmaxf(v[8 * kc + c] + bias[8 * kc + c], 0.f));
                        }
                        const uint4 val = reinterpret_cast<const uint4 *>(o)[kc];
                        if (a.y) {
                            store_rp(a.y, plane + (long long)(x + 1) * 8, AC_BC_ONLY(lim, ) val);
                            if (x == 0)
                                store_rp(a.y, plane + (long long)(a.nx + 1) * 8, AC_BC_ONLY(lim, ) val);
                            if (x == a.nx - 1) store_rp(a.y, plane, AC_BC_ONLY(lim, ) val);
                        }
                    }
                } else {
                    const long long p = AC_BC(((long long)z * a.ny + sg.y) * a.nx + x,
                                              (long long)a.nx * a.ny * a.nz, AC_BC_CONV_OUT);
#pragma unroll
                    for (int c = 0; c < COUT; ++c) {
                        const float val = a.out_scale[c] * (v[c] + bias[c]);
                        a.out[c][p] = val;
                        const float m = fabsf(val);  // exact: the max needs no wider type
                        gm = (m > gm || m != m) ? m : gm;
                    }
                }
            }
        }
        if (!ok && lane == 0) atomicExch(a.err, 1u);
        if (EPI == EPI_SCALED_F32 && a.gmax) {
            unsigned long long bits = (unsigned long long)__double_as_longlong((double)gm);
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long other = __shfl_xor_sync(0xffffffffu, bits, o);
                bits = other > bits ? other : bits;
            }
            if (lane == 0) atomicMax(a.gmax, bits);
        }
    }
    tc_fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, TCOLS);
}

// ---- paired CTAs: tcgen05 with cta_group::2 (M = 256 over two SMs) ---------
//
// A cluster of two CTAs computes two neighbouring columns of one z-chunk in
// lockstep.  Each CTA stages its own column's slices and holds one N-half of
// the kz-stacked weights; the leader (cluster rank 0) issues every MMA with
// cta_group::2, so one instruction covers 256 cells (128 per CTA, each CTA's
// rows landing in its own TMEM) and the per-SM instruction count halves.
// Synchronisation across the pair: the peer's TMA copies complete on the
// leader's slot barrier (cp.async.bulk.tensor .cta_group::2 with the leader's
// barrier), commits are multicast to both CTAs' barriers, and the peer's
// epilogue warps arrive remotely on the leader's TMEM-block barrier.
// Every MMA window spans three TMEM blocks (N = 3 NB): tile t of a segment owns
// block t + 2 and blocks 0, 1, L + 2, L + 3 take the contributions meant for
// tiles outside the segment, which are never read; all segments have the same
// length L (the last z-chunk overlaps the one before it), so those spare
// blocks never hold a real tile.
constexpr int PZC = 12;            // tiles per column segment (L), at most
constexpr int PBLK = PZC + 4;      // TMEM blocks per CTA

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;\n" : "=r"(r));
    return r;
}
// Shared-memory address of the same variable in the leader CTA (cluster window).
__device__ __forceinline__ uint32_t leader_addr(const void *p) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, 0;\n" : "=r"(r) : "r"(smem_u32(p)));
    return r;
}
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n"
                 "barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_alloc2(uint32_t *dst, unsigned ncols) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(dst)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc2(uint32_t taddr, unsigned ncols) {
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols)
                 : "memory");
}
// Paired MMA (accumulating), issued by one elected lane of the leader's converged warp.
__device__ __forceinline__ void mma2_bf16_elect(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                                uint32_t idesc) {
    asm volatile(
        "{\n .reg .pred p, e;\n .reg .b32 r;\n elect.sync r|e, 0xffffffff;\n setp.ne.u32 p, 1, 0;\n"
        " @e tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc)
        : "memory");
}
// Arrive on the barrier at `bar`'s offset in both CTAs once the leader's MMAs so
// far are done (one elected lane).
__device__ __forceinline__ void mma2_commit_elect(uint64_t *bar) {
    const uint16_t mask = 0x3;
    asm volatile(
        "{\n .reg .pred e;\n .reg .b32 r;\n elect.sync r|e, 0xffffffff;\n"
        " @e tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
        " [%0], %1;\n}\n" ::"r"(smem_u32(bar)),
        "h"(mask)
        : "memory");
}
// Tiled TMA load into this CTA's shared memory, completing on a barrier given by
// its cluster-window address (the leader's).
__device__ __forceinline__ void tma2_load_5d(void *dst, const CUtensorMap *map, uint32_t bar_cluster,
                                             int c0, int c1, int c2, int c3, int c4) {
    asm volatile(
        "cp.async.bulk.tensor.5d.cta_group::2.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5, %6, %7}], [%2];\n" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar_cluster), "r"(c0), "r"(c1), "r"(c2), "r"(c3),
        "r"(c4)
        : "memory");
}
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t bar_cluster) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];\n" ::"r"(bar_cluster)
                 : "memory");
}

// Column pair segment h (chunk-major over column pairs): this CTA's column is
// 2 pc + rank; when the column count is odd the last pair's second CTA repeats
// column ncols - 1 and writes nothing.  Every segment has a.zc tiles; the last
// chunk starts at nz - zc, and only its tiles from chunk * zc on are written
// (those before it belong to the chunk before).
struct PairSegment {
    Segment s;
    int zw;      // first z this CTA writes
    bool write;  // false: duplicate column
};

__device__ __forceinline__ PairSegment pair_segment_of(long long h, const ConvTcArgs &a, int segs,
                                                       uint32_t rank) {
    const int ncols = a.ny * segs;
    const int pcols = (ncols + 1) / 2;
    const int chunk = (int)(h / pcols);
    const int pc = (int)(h - (long long)chunk * pcols);
    int col = 2 * pc + (int)rank;
    PairSegment p;
    p.write = col < ncols;
    col = p.write ? col : ncols - 1;
    p.s.y = col / segs;
    p.s.seg = col - p.s.y * segs;
    p.zw = chunk * a.zc;
    p.s.z0 = p.zw + a.zc <= a.nz ? p.zw : a.nz - a.zc;
    p.s.len = a.zc;
    return p;
}

// Shared memory of one CTA of a pair: its half of the weight image and the ring.
constexpr int PNBUF = 6;
__host__ __device__ constexpr size_t pair_smem_bytes(int cin) {
    return (size_t)w_bytes(cin, 32) / 2 + (size_t)PNBUF * 3 * row_bytes(cin);
}

// The paired kernel.  Same slice numbering, ring and weight-image order as
// conv_tc_kernel, with these differences: the image is split by kz-stack rows,
// rows [r 3NB/2, (r+1) 3NB/2) in CTA r; slice j of a segment always issues the
// full window, N = 3 NB at TMEM block j (blocks j .. j+2 = tiles j-2 .. j);
// the barriers live in both CTAs but only these phases are used:
//   leader full[b]  : expect_tx of both CTAs' slice bytes; both CTAs' TMA land on it;
//   empty[b], accf[k], fin : multicast commits, waited on locally in each CTA;
//   leader acce[k]  : 8 arrivals, the four epilogue warps of each CTA;
//   wbar            : this CTA's weight half landed (checked before the cluster
//                     barrier that precedes the first MMA).
template <int CIN, int COUT, int EPI>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(THREADS, 1)
    conv_tc_pair_kernel(const __grid_constant__ CUtensorMap xmap, const ConvTcArgs a) {
    static_assert(EPI != EPI_MASK_BF16, "the paired kernel has no mask epilogue");
    // N = 3 NB must be a multiple of 32 for cta_group::2, so the stack always has
    // 32 rows per kz (zero weights past COUT); the epilogue reads NR of them
    constexpr int NB = 32;
    constexpr int NR = COUT < 16 ? 16 : COUT;
    constexpr int KC = CIN / 8;
    constexpr bool PAIR = CIN == 8;
    constexpr int NGH = 3 * NB / 16;           // core-matrix rows of this CTA's stack half
    constexpr int ROW = row_bytes(CIN);
    constexpr int SLICE = 3 * ROW;
    constexpr int WH_BYTES = w_bytes(CIN, NB) / 2;
    constexpr uint32_t SLICE_TX = 3 * KC * PLANE;
    constexpr uint32_t TCOLS = PBLK * NB;      // 512 or 256 TMEM columns
    constexpr uint32_t IDESC = idesc_bf16(2 * TM, 3 * NB);
    static_assert((CIN % 16 == 0 || CIN == 8) && COUT % 8 == 0 && COUT <= 32, "shape");
    static_assert(NGH * 16 == 3 * NB && PBLK <= 32, "stack halves, block masks");
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t full[PNBUF], empty[PNBUF], accf[PBLK], acce[PBLK], wbar, fin;
    __shared__ uint32_t tmem_base;
    unsigned char *Ws = smem;
    unsigned char *Ss = smem + WH_BYTES;
    const uint32_t rank = cluster_rank();
    const bool leader = rank == 0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int segs = (a.nx + TM - 1) / TM;
    const int ncols = a.ny * segs;
    const long long nseg = (long long)((a.nz + a.zc - 1) / a.zc) * ((ncols + 1) / 2);
    const long long pair0 = blockIdx.x >> 1, npairs = gridDim.x >> 1;
    const int L = a.zc;

    if (warp == 0) tmem_alloc2(&tmem_base, TCOLS);
    if (threadIdx.x == 128) {
        for (int b = 0; b < PNBUF; ++b) {
            mbar_init(&full[b], 1);
            mbar_init(&empty[b], 1);
        }
        for (int k = 0; k < PBLK; ++k) {
            mbar_init(&accf[k], 1);
            mbar_init(&acce[k], 8);
        }
        mbar_init(&wbar, 1);
        mbar_init(&fin, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        mbar_expect_tx(&wbar, WH_BYTES);
        bulk_load(Ws, reinterpret_cast<const unsigned char *>(a.w) + rank * WH_BYTES, WH_BYTES, &wbar);
    }
    __syncthreads();  // TMEM address published
    tc_fence_after_sync();
    const uint32_t tmem = tmem_base;
    if (warp < 4) {  // every accumulator block starts at zero
        for (int k = 0; k < PBLK; ++k) tmem_zero<NB>(tmem + ((uint32_t)(warp * 32) << 16) + k * NB);
        tc_fence_before_sync();
    }
    if (threadIdx.x == 128 && !mbar_wait(&wbar, 0)) atomicExch(a.err, 1u);
    // both CTAs: barriers initialised, TMEM zeroed, weight halves landed
    cluster_sync();
    tc_fence_after_sync();

    if (warp == 4) {
        if (lane == 0) {  // ---- TMA producer (both CTAs; completions land on the leader's full[b])
            long long s = 0;
            bool ok = true;
            for (long long h = pair0; h < nseg && ok; h += npairs) {
                const Segment sg = pair_segment_of(h, a, segs, rank).s;
                for (int j = 0; j < L + 2; ++j, ++s) {
                    const int b = (int)(s % PNBUF);
                    const long long k = s / PNBUF;
                    if (k > 0 && !mbar_wait(&empty[b], (unsigned)((k - 1) & 1))) {
                        ok = false;
                        break;
                    }
                    if (leader) mbar_expect_tx(&full[b], 2 * SLICE_TX);
                    const uint32_t fb = leader_addr(&full[b]);
                    const int z = wrapi(sg.z0 + j - 1, a.nz);
                    unsigned char *dst = Ss + b * SLICE;
#pragma unroll
                    for (int r = 0; r < 3; ++r)
                        tma2_load_5d(dst + r * ROW, &xmap, fb, 0, sg.seg * (TM / 8), 0,
                                     wrapi(sg.y + r - 1, a.ny), z);
                }
            }
            if (!ok) atomicExch(a.err, 1u);
            // no copy may be in flight when either CTA exits: the leader waits for
            // each buffer's last fill (both CTAs' bytes) before the final cluster barrier
            if (leader)
                for (int b = 0; b < PNBUF; ++b)
                    if (s > b) mbar_wait(&full[b], (unsigned)(((s - 1 - b) / PNBUF) & 1));
        }
    } else if (warp == 5) {
        if (leader) {  // ---- MMA issuer: the leader's whole warp, one elected lane issues
            static_assert(GROUP == 3, "the combined wait tests six barriers");
            bool ok = true;
            long long s = 0;
            // bit k of `used`: block k has held a tile; bit k of `par`: parity of their count
            uint32_t used = 0, par = 0;
            const uint64_t b0 = smem_desc(smem_u32(Ws), NGH * CORE, CORE);
            for (long long h = pair0; h < nseg && ok; h += npairs) {
                for (int j = 0; j < L + 2; ++j, ++s) {
                    const int b = (int)(s % PNBUF);
                    if (j % GROUP == 0) {
                        uint32_t addr[2 * GROUP];
                        unsigned want[2 * GROUP];
                        uint32_t pending = 0;
#pragma unroll
                        for (int q = 0; q < GROUP; ++q) {
                            const long long sq = s + q;
                            const int jq = j + q;
                            const int kq = jq < L ? jq + 2 : 0;  // block tile jq opens
                            addr[2 * q] = smem_u32(&full[sq % PNBUF]);
                            want[2 * q] = (unsigned)((sq / PNBUF) & 1);
                            addr[2 * q + 1] = smem_u32(&acce[kq]);
                            want[2 * q + 1] = ((par >> kq) & 1u) ^ 1u;
                            if (jq < L + 2) pending |= 1u << (2 * q);
                            if (jq < L && ((used >> kq) & 1u)) pending |= 1u << (2 * q + 1);
                        }
                        ok = mbar_wait6_warp(addr, want, pending);
                        if (!ok) break;
                        tc_fence_after_sync();
                    }
                    if (j < L) {  // tile j opens in block j + 2
                        used |= 1u << (j + 2);
                        par ^= 1u << (j + 2);
                    }
                    const uint32_t sbase = smem_u32(Ss + b * SLICE);
                    const uint32_t dtm = tmem + (uint32_t)(j * NB);
                    if constexpr (PAIR) {
                        const uint64_t a0 = smem_desc(sbase, 0, CORE);
#pragma unroll
                        for (int p = 0; p < 5; ++p) {
                            const int ta0 = pair_tap(p, 0), tb0 = pair_tap(p, 1);
                            const uint32_t off = (ta0 / 3) * ROW + (ta0 % 3) * 16;
                            const uint32_t lbo = (tb0 / 3) * ROW + (tb0 % 3) * 16 - off;
                            const uint64_t ad = a0 + (off >> 4) + ((uint64_t)(lbo >> 4) << 16);
                            const uint64_t bd = b0 + ((2 * p * NGH * CORE) >> 4);
                            mma2_bf16_elect(dtm, ad, bd, IDESC);
                        }
                    } else {
                        const uint64_t a0 = smem_desc(sbase, PLANE, CORE);
#pragma unroll
                        for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                            for (int dx = 0; dx < 3; ++dx)
#pragma unroll
                                for (int kk = 0; kk < CIN / 16; ++kk) {
                                    const int dyx = dy * 3 + dx;
                                    const uint64_t ad = a0 + ((dy * ROW + dx * 16 + kk * 2 * PLANE) >> 4);
                                    const uint64_t bd = b0 + (((dyx * KC + 2 * kk) * NGH * CORE) >> 4);
                                    mma2_bf16_elect(dtm, ad, bd, IDESC);
                                }
                    }
                    mma2_commit_elect(&empty[b]);
                    if (j >= 2) mma2_commit_elect(&accf[j]);  // block j: tile j-2 has had its third slice
                }
            }
            if (!ok && lane == 0) atomicExch(a.err, 1u);
            // no MMA may be in flight when TMEM is freed: a final commit covers all
            mma2_commit_elect(&fin);
            mbar_wait(&fin, 0);
        } else if (lane == 0) {
            // the peer: the final commit's arrival on its own fin is the last write
            // the leader's MMAs make into this CTA; it must land before the CTA exits
            if (!mbar_wait(&fin, 0)) atomicExch(a.err, 1u);
        }
    } else {  // ---- epilogue: warps 0-3 of each CTA, its TMEM lanes 32 warp .. 32 warp + 31
        float bias[COUT];
#pragma unroll
        for (int c = 0; c < COUT; ++c) bias[c] = a.bias[c];
        float gm = 0.f;
        uint32_t par = 0;  // bit k: parity of the tiles block k has held so far
        bool ok = true;
        for (long long h = pair0; h < nseg && ok; h += npairs) {
            const PairSegment ps = pair_segment_of(h, a, segs, rank);
            const Segment &sg = ps.s;
            const int x = sg.seg * TM + warp * 32 + lane;
            for (int i = 0; i < L; ++i) {
                const int kb = i + 2;
                ok = __all_sync(0xffffffffu, mbar_wait(&accf[kb], (par >> kb) & 1u));
                par ^= 1u << kb;
                if (!ok) break;
                tc_fence_after_sync();
                const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(kb * NB);
                float v[NR];
                if constexpr (NR == 32)
                    tmem_ld32(taddr, v);
                else
                    tmem_ld16(taddr, v);
                tmem_zero<NR>(taddr);  // columns past NR only ever receive zero weights
                tc_fence_before_sync();
                __syncwarp();
                if (lane == 0) mbar_arrive_cluster(leader_addr(&acce[kb]));
                const int z = sg.z0 + i;
                if (!ps.write || z < ps.zw || x >= a.nx) continue;
                if (EPI == EPI_RELU_BF16) {
                    __align__(16) bf16 o[COUT];
                    AC_BC_ONLY(const long long lim =
                                   (long long)rp_cells(a.nx) * a.ny * a.nz * COUT;)
#pragma unroll
                    for (int kc = 0; kc < COUT / 8; ++kc) {
                        const long long plane =
                            ((((long long)z * a.ny + sg.y) * (COUT / 8) + kc) * rp_cells(a.nx)) * 8;
#pragma unroll
                        for (int c = 0; c < 8; ++c)
                            o[8 * kc + c] =
                                __float2bfloat16_rn(fmaxf(v[8 * kc + c] + bias[8 * kc + c], 0.f));
                        const uint4 val = reinterpret_cast<const uint4 *>(o)[kc];
                        if (a.y) {
                            store_rp(a.y, plane + (long long)(x + 1) * 8, AC_BC_ONLY(lim, ) val);
                            if (x == 0)
                                store_rp(a.y, plane + (long long)(a.nx + 1) * 8, AC_BC_ONLY(lim, ) val);
                            if (x == a.nx - 1) store_rp(a.y, plane, AC_BC_ONLY(lim, ) val);
                        }
                    }
                } else {
                    const long long p = AC_BC(((long long)z * a.ny + sg.y) * a.nx + x,
                                              (long long)a.nx * a.ny * a.nz, AC_BC_CONV_OUT);
#pragma unroll
                    for (int c = 0; c < COUT; ++c) {
                        const float val = a.out_scale[c] * (v[c] + bias[c]);
                        a.out[c][p] = val;
                        const float m = fabsf(val);  // exact: the max needs no wider type
                        gm = (m > gm || m != m) ? m : gm;
                    }
                }
            }
        }
        if (!ok && lane == 0) atomicExch(a.err, 1u);
        if (EPI == EPI_SCALED_F32 && a.gmax) {
            unsigned long long bits = (unsigned long long)__double_as_longlong((double)gm);
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long other = __shfl_xor_sync(0xffffffffu, bits, o);
                bits = other > bits ? other : bits;
            }
            if (lane == 0) atomicMax(a.gmax, bits);
        }
    }
    // the leader's MMAs have finished (it waited on fin), every remote arrival
    // and every copy into either CTA has landed: TMEM can go
    tc_fence_before_sync();
    cluster_sync();
    if (warp == 0) tmem_dealloc2(tmem, TCOLS);
}

// Weight image for conv_tc_kernel from binary32 W[cout][cin_real][27] (tap =
// 9 kz + 3 ky + kx); nb = accumulator columns per tile (COUT padded to 16 or
// 32); cin = 8 gives the tap-pair image.  Only the core-matrix rows ng_lo ..
// ng_lo + ng_cnt - 1 of the kz stack are written, as an image of their own
// (ng_cnt = 3 nb / 8 for the whole stack; the paired kernel takes the two
// halves one after the other).
__global__ void conv_tc_prep_kernel(const float *__restrict__ W, int cout, int cin_real, int cin,
                                    int nb, int ng_lo, int ng_cnt, bf16 *__restrict__ img) {
    const int KC = cin / 8;
    const bool pair = cin == 8;
    const int total = (pair ? 10 : 9 * KC) * ng_cnt * 64;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int c = i & 7, r = (i >> 3) & 7;
        const int rest = i >> 6;  // kq * ng_cnt + (ng - ng_lo)
        const int ng = ng_lo + rest % ng_cnt;
        const int kq = rest / ng_cnt;
        int dyx, ci;
        bool live = true;
        if (pair) {
            const int p = kq >> 1, h = kq & 1;
            dyx = pair_tap(p, h);
            ci = c;
            live = !(p == 4 && h == 0);
        } else {
            dyx = kq / KC;
            ci = 8 * (kq % KC) + c;
        }
        const int row = 8 * ng + r;
        const int kz = 2 - row / nb, co = row % nb;
        const float v = (live && co < cout && ci < cin_real)
                            ? W[((long long)co * cin_real + ci) * 27 + kz * 9 + dyx]
                            : 0.f;
        img[i] = __float2bfloat16_rn(v);
    }
}

}  // namespace tc
}  // namespace ac
