// Domain decomposition with halo exchange (Sec. 3.2-3.3): the periodic grid is
// split into px x py x pz subdomains, each held with a radius-3 halo; every
// substep packs the outbound halo segments, delivers them as messages, unpacks
// them into the neighbours' halos and updates the outer segments, while the
// inner segment (no halo read) is updated concurrently on another stream.
//
// Here all subdomains live on one device: a message is a device-local copy
// between packed buffers, so the pipeline -- and its result, bitwise equal to
// the undecomposed binary64 and binary32 padded-layout substep -- is what a
// multi-device run would exchange, without a second device.
//
// Segments (Sec. 3.3): 6 sides and 12 edges.  The 8 corners are not exchanged:
// no point of the Eq. 13 stencil lies off the axes and face diagonals, so no
// corner halo cell is ever read.  A segment in direction d is identified by d
// (the message tag); its cells in the receiver's halo map onto the sender's
// interior by s' = ((s - r) mod n') + r per axis.
//
// Mapping of subdomains to devices (Sec. 3.3): Z-order, the subdomain
// coordinates sorted by their Morton codes (bits of x, y, z interleaved, x
// lowest); for a power-of-two count the partition P = morton^-1(count - 1) +
// (1, 1, 1) of the paper.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "substep.cuh"

namespace ac {

constexpr int DC_SEGS = 18;  // 6 sides + 12 edges

// Direction vectors of the segments: sides first (x-, x+, y-, y+, z-, z+), then
// the edges in lexicographic order of d.
static void dc_dirs(int dirs[DC_SEGS][3]) {
    int k = 0;
    for (int a = 0; a < 3; ++a)
        for (int sgn = -1; sgn <= 1; sgn += 2) {
            dirs[k][0] = dirs[k][1] = dirs[k][2] = 0;
            dirs[k][a] = sgn;
            ++k;
        }
    for (int z = -1; z <= 1; ++z)
        for (int y = -1; y <= 1; ++y)
            for (int x = -1; x <= 1; ++x) {
                const int nz = (x != 0) + (y != 0) + (z != 0);
                if (nz != 2) continue;
                dirs[k][0] = x;
                dirs[k][1] = y;
                dirs[k][2] = z;
                ++k;
            }
}

static unsigned long long morton3(int x, int y, int z) {
    unsigned long long m = 0;
    for (int b = 0; b < 21; ++b) {
        m |= (unsigned long long)((x >> b) & 1) << (3 * b);
        m |= (unsigned long long)((y >> b) & 1) << (3 * b + 1);
        m |= (unsigned long long)((z >> b) & 1) << (3 * b + 2);
    }
    return m;
}

// Coordinates of the subdomain with Z-order position `rank` in a p grid.
static int dc_coord(const int p[3], int rank, int c[3]) {
    const int n = p[0] * p[1] * p[2];
    if (rank < 0 || rank >= n) return AC_ERR_ARG;
    // the rank-th smallest Morton code among the grid's coordinates
    std::vector<unsigned long long> codes;
    codes.reserve(n);
    for (int z = 0; z < p[2]; ++z)
        for (int y = 0; y < p[1]; ++y)
            for (int x = 0; x < p[0]; ++x) codes.push_back(morton3(x, y, z));
    std::vector<unsigned long long> sorted = codes;
    std::sort(sorted.begin(), sorted.end());
    const unsigned long long want = sorted[rank];
    for (int z = 0; z < p[2]; ++z)
        for (int y = 0; y < p[1]; ++y)
            for (int x = 0; x < p[0]; ++x)
                if (morton3(x, y, z) == want) {
                    c[0] = x;
                    c[1] = y;
                    c[2] = z;
                    return AC_OK;
                }
    return AC_ERR_ARG;
}

static int dc_valid_p(const int p[3]) {
    if (!p) return 0;
    for (int a = 0; a < 3; ++a)
        if (p[a] < 1 || p[a] > 64) return 0;
    return p[0] * p[1] * p[2] <= 512;
}

// One subdomain on the device.
struct DcSub {
    int coord[3];
    int off[3];      // global index of its first interior cell
    Geom g;          // padded geometry of the local grid
    void *state[2][NF];
    void *w[NF];
    double2 *ftab;   // its forcing tables [nx' | ny' | nz'] (double2, then float2)
};

// One message: the cells of segment d of subdomain `src` (its interior box) go
// to the halo box of subdomain `dst`; packed as 8 contiguous fields of `cells`.
struct DcMsg {
    int src, dst;
    int sb0[3];  // source box origin, padded coordinates of src
    int db0[3];  // destination box origin, padded coordinates of dst
    int ext[3];
    long long cells;
    long long off;  // element offset of the packed block in the message buffers
};

}  // namespace ac

using namespace ac;

struct ac_decomp {
    ac_grid grid;
    ac_params params;
    int p[3];
    int nsub;
    int nloc[3];
    StencilCoefs coefs;
    PhysConsts phys;
    int elem_f, elem_w;
    cudaStream_t stream;   // the caller's stream: updates
    cudaStream_t comm;     // pack, messages, unpack (higher priority)
    cudaEvent_t ev_start, ev_unpacked;
    // the outer slabs of all subdomains run on DC_OUTER streams at once (each slab
    // alone fills the GPU poorly); the caller's stream waits for all of them
    static constexpr int DC_OUTER = 4;
    cudaStream_t outer[DC_OUTER];
    cudaEvent_t ev_outer[DC_OUTER];
    std::vector<DcSub> sub;
    std::vector<DcMsg> msgs;
    DcMsg *msgs_dev;
    void **ptrs_dev;       // [nsub][2][NF] state pointers, for the pack/unpack kernels
    void *sendbuf, *recvbuf;
    long long msg_elems;
    void *block;           // all subdomain arrays
    double *stage;         // host<->device staging of one subdomain field (binary64)
    size_t stage_elems;
    int cur;
    int next_s;
    unsigned long long step;
    int overlap;
    unsigned long long launches;
    int force_k[3];
    double force_e[3], force_phi;
    unsigned long long ftab_step;
    int ftab_valid;
};

namespace ac {

// Pack (or unpack) every message: one CTA row per message (blockIdx.y), the
// message's 8 fields x cells over blockIdx.x and the threads.  Pack reads the
// source subdomain's interior box into the packed buffer; unpack writes the
// packed buffer into the destination subdomain's halo box.
template <typename T, bool PACK>
__global__ void dc_pack_kernel(const DcMsg *msgs, void *const *ptrs, int cur, const Geom *geoms,
                               T *buf) {
    const DcMsg m = msgs[blockIdx.y];
    const int sd = PACK ? m.src : m.dst;
    const Geom g = geoms[sd];
    const int *b0 = PACK ? m.sb0 : m.db0;
    const long long total = NF * m.cells;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int q = (int)(t / m.cells);
        const long long c = t - q * m.cells;
        const int ex = m.ext[0], ey = m.ext[1];
        const int k = (int)(c / ((long long)ex * ey));
        const long long rem = c - (long long)k * ex * ey;
        const int j = (int)(rem / ex);
        const int i = (int)(rem - (long long)j * ex);
        const long long o =
            (long long)(b0[2] + k) * g.pxy + (long long)(b0[1] + j) * g.px + (b0[0] + i);
        T *arr = static_cast<T *>(ptrs[(sd * 2 + cur) * NF + q]);
        const long long bo = m.off + t;
        if (PACK)
            buf[bo] = arr[AC_BC(o, g.elems, AC_BC_STENCIL)];
        else
            arr[AC_BC(o, g.elems, AC_BC_STENCIL)] = buf[bo];
    }
}

// Message delivery on one device: every message's packed block is copied from
// the sender's slot of the send buffer to the receiver's slot of the receive
// buffer (the slots coincide: one slot per message).
template <typename T>
__global__ void dc_deliver_kernel(const T *__restrict__ send, T *__restrict__ recv, long long n) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x)
        recv[t] = send[t];
}

// Forcing tables of one subdomain: the global tables' entries at its global
// indices, e^{i 2 pi k_a (off_a + i) / n_a} (phi folded into z), computed with
// the same operations as the global table so that entries agree bitwise.
__global__ void dc_forcing_table_kernel(int nx, int ny, int nz, int ox, int oy, int oz, int gnx,
                                        int gny, int gnz, int kx, int ky, int kz, double cphi,
                                        double sphi, double2 *tab) {
    const int total = nx + ny + nz;
    float2 *tabf = reinterpret_cast<float2 *>(tab + total);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        int n, kk, i;
        if (t < nx) {
            n = gnx; kk = kx; i = ox + t;
        } else if (t < nx + ny) {
            n = gny; kk = ky; i = oy + t - nx;
        } else {
            n = gnz; kk = kz; i = oz + t - nx - ny;
        }
        long long m = ((long long)kk * i) % n;
        if (m < 0) m += n;
        double s, c;
        sincospi(2.0 * (double)m / (double)n, &s, &c);
        if (t >= nx + ny) {
            const double c2 = c * cphi - s * sphi;
            const double s2 = s * cphi + c * sphi;
            c = c2;
            s = s2;
        }
        tab[t] = make_double2(c, s);
        tabf[t] = make_float2((float)c, (float)s);
    }
}

template <typename R, typename W>
static cudaError_t dc_update_box(ac_decomp *d, int si, const Box &box, double alpha,
                                 double beta, double dt, int s, cudaStream_t st) {
    for (int a = 0; a < 3; ++a)
        if (box.b1[a] <= box.b0[a]) return cudaSuccess;
    const DcSub &sb = d->sub[si];
    SubstepArgs<R, W> a;
    a.g = sb.g;
    for (int q = 0; q < NF; ++q) {
        a.fin[q] = static_cast<const R *>(sb.state[d->cur][q]);
        a.fout[q] = static_cast<R *>(sb.state[1 - d->cur][q]);
        a.w[q] = static_cast<W *>(sb.w[q]);
    }
    a.k = to_dev<R>(d->coefs, d->phys);
    a.alpha = (W)alpha;
    a.beta = (W)beta;
    a.dt = (W)dt;
    a.s0 = s == 0;
    a.force_on = d->params.force_amp != 0.0;
    const long long ntab = (long long)sb.g.nx + sb.g.ny + sb.g.nz;
    if (sizeof(R) == 8)
        a.ftab = reinterpret_cast<const typename Vec2<R>::type *>(sb.ftab);
    else
        a.ftab = reinterpret_cast<const typename Vec2<R>::type *>(sb.ftab + ntab);
    for (int m = 0; m < 3; ++m) a.amp_e[m] = (R)(d->params.force_amp * d->force_e[m]);
    a.cfl_max = nullptr;
    const int ex = box.b1[0] - box.b0[0], ey = box.b1[1] - box.b0[1], ez = box.b1[2] - box.b0[2];
    const bool flat = ex < 32;  // a slab a few cells thin in x
    const dim3 block = flat ? dim3(128, 1, 1) : dim3(32, 4, 1);
    const unsigned gx = flat ? (unsigned)(((long long)ex * ey + 127) / 128) : (unsigned)((ex + 31) / 32);
    const unsigned gy = flat ? 1u : (unsigned)((ey + 3) / 4);
    int zc = (int)(((long long)gx * gy * ez) / (8 * 152));
    zc = zc < 1 ? 1 : (zc > 16 ? 16 : zc);
    a.zchunk = zc;
    const dim3 grid(gx, gy, (ez + zc - 1) / zc);
    const bool ext = d->phys.ext();
    if (flat) {
        if (ext) substep_box_kernel<R, W, 3, true, true><<<grid, block, 0, st>>>(a, box);
        else substep_box_kernel<R, W, 3, false, true><<<grid, block, 0, st>>>(a, box);
    } else {
        if (ext) substep_box_kernel<R, W, 3, true, false><<<grid, block, 0, st>>>(a, box);
        else substep_box_kernel<R, W, 3, false, false><<<grid, block, 0, st>>>(a, box);
    }
    d->launches++;
    return cudaGetLastError();
}

static cudaError_t dc_update(ac_decomp *d, int si, const Box &box, double alpha, double beta,
                             double dt, int s, cudaStream_t st) {
    if (d->params.precision == AC_FP64)
        return dc_update_box<double, double>(d, si, box, alpha, beta, dt, s, st);
    if (d->params.precision == AC_FP32)
        return dc_update_box<float, float>(d, si, box, alpha, beta, dt, s, st);
    return dc_update_box<float, double>(d, si, box, alpha, beta, dt, s, st);
}

template <bool PACK>
static cudaError_t dc_pack(ac_decomp *d, void *buf, cudaStream_t st, const Geom *geoms_dev) {
    const int nm = (int)d->msgs.size();
    long long maxc = 0;
    for (const DcMsg &m : d->msgs) maxc = m.cells > maxc ? m.cells : maxc;
    long long bx = (NF * maxc + 255) / 256;
    if (bx > 64) bx = 64;
    const dim3 grid((unsigned)bx, nm);
    if (d->elem_f == 8)
        dc_pack_kernel<double, PACK><<<grid, 256, 0, st>>>(d->msgs_dev, d->ptrs_dev, d->cur,
                                                           geoms_dev, static_cast<double *>(buf));
    else
        dc_pack_kernel<float, PACK><<<grid, 256, 0, st>>>(d->msgs_dev, d->ptrs_dev, d->cur,
                                                          geoms_dev, static_cast<float *>(buf));
    d->launches++;
    return cudaGetLastError();
}

}  // namespace ac

// Per-subdomain geometries follow the message table on the device.
static const Geom *dc_geoms_dev(const ac_decomp *d) {
    return reinterpret_cast<const Geom *>(d->msgs_dev + d->msgs.size());
}

extern "C" int ac_decomp_partition(int count, int p[3]) {
    if (!p || count < 1 || count > 512 || (count & (count - 1))) return AC_ERR_ARG;
    // P = morton^-1(count - 1) + (1, 1, 1)
    const unsigned v = (unsigned)(count - 1);
    int c[3] = {0, 0, 0};
    for (int b = 0; b < 10; ++b)
        for (int a = 0; a < 3; ++a) c[a] |= (int)((v >> (3 * b + a)) & 1u) << b;
    for (int a = 0; a < 3; ++a) p[a] = c[a] + 1;
    return AC_OK;
}

extern "C" int ac_decomp_coord(const int p[3], int rank, int coord[3]) {
    if (!dc_valid_p(p) || !coord) return AC_ERR_ARG;
    return dc_coord(p, rank, coord);
}

extern "C" int ac_decomp_segment(const int nloc[3], int seg, int dir[3], int src_b0[3],
                                 int dst_b0[3], int ext[3]) {
    if (!nloc || !dir || !src_b0 || !dst_b0 || !ext || seg < 0 || seg >= DC_SEGS)
        return AC_ERR_ARG;
    for (int a = 0; a < 3; ++a)
        if (nloc[a] < 2 * R) return AC_ERR_ARG;
    int dirs[DC_SEGS][3];
    dc_dirs(dirs);
    for (int a = 0; a < 3; ++a) {
        const int da = dirs[seg][a], n = nloc[a];
        dir[a] = da;
        // receiver's halo box (padded coordinates: interior starts at R)
        dst_b0[a] = da < 0 ? 0 : (da > 0 ? R + n : R);
        ext[a] = da == 0 ? n : R;
        // the sender (receiver + d) supplies its interior cells s' = ((s - r) mod n) + r
        src_b0[a] = ((dst_b0[a] - R) % n + n) % n + R;
    }
    return AC_OK;
}

static void dc_free(ac_decomp *d) {
    if (d->block) cudaFree(d->block);
    if (d->sendbuf) cudaFree(d->sendbuf);
    if (d->recvbuf) cudaFree(d->recvbuf);
    if (d->msgs_dev) cudaFree(d->msgs_dev);
    if (d->ptrs_dev) cudaFree(d->ptrs_dev);
    if (d->stage) cudaFree(d->stage);
    for (DcSub &s : d->sub)
        if (s.ftab) cudaFree(s.ftab);
    if (d->comm) cudaStreamDestroy(d->comm);
    if (d->ev_start) cudaEventDestroy(d->ev_start);
    if (d->ev_unpacked) cudaEventDestroy(d->ev_unpacked);
    for (int k = 0; k < ac_decomp::DC_OUTER; ++k) {
        if (d->outer[k]) cudaStreamDestroy(d->outer[k]);
        if (d->ev_outer[k]) cudaEventDestroy(d->ev_outer[k]);
    }
}

#define DCK(call)                                       \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return ac_report_cuda(e_); \
    } while (0)

static int dc_setup(ac_decomp *d) {
    const int nsub = d->nsub;
    d->sub.resize(nsub);
    const Geom g = make_geom(d->nloc[0], d->nloc[1], d->nloc[2], AC_LAYOUT_PADDED);
    const size_t bf = ((size_t)g.elems * d->elem_f + 255) / 256 * 256;
    const size_t bw = ((size_t)g.elems * d->elem_w + 255) / 256 * 256;
    const size_t per = 2 * NF * bf + NF * bw;
    DCK(cudaMalloc(&d->block, per * nsub));
    DCK(cudaMemsetAsync(d->block, 0, per * nsub, d->stream));
    int dirs[DC_SEGS][3];
    dc_dirs(dirs);
    for (int r = 0; r < nsub; ++r) {
        DcSub &s = d->sub[r];
        memset(&s, 0, sizeof s);
        int rc = dc_coord(d->p, r, s.coord);
        if (rc) return rc;
        for (int a = 0; a < 3; ++a) s.off[a] = s.coord[a] * d->nloc[a];
        s.g = g;
        char *base = static_cast<char *>(d->block) + per * r;
        for (int b = 0; b < 2; ++b)
            for (int q = 0; q < NF; ++q) s.state[b][q] = base + (b * NF + q) * bf;
        for (int q = 0; q < NF; ++q) s.w[q] = base + 2 * NF * bf + q * bw;
        DCK(cudaMalloc(&s.ftab, (size_t)(g.nx + g.ny + g.nz) * (sizeof(double2) + sizeof(float2))));
    }
    // rank of each coordinate
    std::vector<int> rank_of(nsub);
    for (int r = 0; r < nsub; ++r) {
        const int *c = d->sub[r].coord;
        rank_of[(c[2] * d->p[1] + c[1]) * d->p[0] + c[0]] = r;
    }
    // messages: receiver r, direction d: sender = r + d (periodic in the p grid)
    long long off = 0;
    for (int r = 0; r < nsub; ++r) {
        for (int k = 0; k < DC_SEGS; ++k) {
            DcMsg m;
            int dir[3];
            ac_decomp_segment(d->nloc, k, dir, m.sb0, m.db0, m.ext);
            int c[3];
            for (int a = 0; a < 3; ++a)
                c[a] = ((d->sub[r].coord[a] + dir[a]) % d->p[a] + d->p[a]) % d->p[a];
            m.src = rank_of[(c[2] * d->p[1] + c[1]) * d->p[0] + c[0]];
            m.dst = r;
            m.cells = (long long)m.ext[0] * m.ext[1] * m.ext[2];
            m.off = off;
            off += NF * m.cells;
            d->msgs.push_back(m);
        }
    }
    d->msg_elems = off;
    const size_t mb = (size_t)off * d->elem_f;
    DCK(cudaMalloc(&d->sendbuf, mb));
    DCK(cudaMalloc(&d->recvbuf, mb));
    const size_t tab_bytes = d->msgs.size() * sizeof(DcMsg) + nsub * sizeof(Geom);
    DCK(cudaMalloc(&d->msgs_dev, tab_bytes));
    std::vector<char> host(tab_bytes);
    memcpy(host.data(), d->msgs.data(), d->msgs.size() * sizeof(DcMsg));
    for (int r = 0; r < nsub; ++r)
        memcpy(host.data() + d->msgs.size() * sizeof(DcMsg) + r * sizeof(Geom), &d->sub[r].g,
               sizeof(Geom));
    DCK(cudaMemcpy(d->msgs_dev, host.data(), tab_bytes, cudaMemcpyHostToDevice));
    std::vector<void *> ptrs((size_t)nsub * 2 * NF);
    for (int r = 0; r < nsub; ++r)
        for (int b = 0; b < 2; ++b)
            for (int q = 0; q < NF; ++q) ptrs[(r * 2 + b) * NF + q] = d->sub[r].state[b][q];
    DCK(cudaMalloc(&d->ptrs_dev, ptrs.size() * sizeof(void *)));
    DCK(cudaMemcpy(d->ptrs_dev, ptrs.data(), ptrs.size() * sizeof(void *), cudaMemcpyHostToDevice));
    int lo = 0, hi = 0;
    DCK(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    DCK(cudaStreamCreateWithPriority(&d->comm, cudaStreamNonBlocking, hi));
    DCK(cudaEventCreateWithFlags(&d->ev_start, cudaEventDisableTiming));
    DCK(cudaEventCreateWithFlags(&d->ev_unpacked, cudaEventDisableTiming));
    for (int k = 0; k < ac_decomp::DC_OUTER; ++k) {
        DCK(cudaStreamCreateWithFlags(&d->outer[k], cudaStreamNonBlocking));
        DCK(cudaEventCreateWithFlags(&d->ev_outer[k], cudaEventDisableTiming));
    }
    const size_t plane = (size_t)d->nloc[0] * d->nloc[1];
    d->stage_elems = plane * d->nloc[2];
    DCK(cudaMalloc(&d->stage, d->stage_elems * sizeof(double)));
    return AC_OK;
}

extern "C" int ac_decomp_init(ac_decomp **out, const ac_grid *grid, const ac_params *params,
                              const int p[3], void *stream) {
    if (!out || !valid_grid(grid) || !valid_params(params) || !dc_valid_p(p)) return AC_ERR_ARG;
    if (grid->layout != AC_LAYOUT_PERIODIC) return AC_ERR_ARG;
    int nloc[3];
    const int n[3] = {grid->nx, grid->ny, grid->nz};
    for (int a = 0; a < 3; ++a) {
        if (n[a] % p[a]) return AC_ERR_ARG;
        nloc[a] = n[a] / p[a];
        if (nloc[a] < 2 * R) return AC_ERR_ARG;  // inner and outer segments need n' >= 2r
    }
    *out = nullptr;
    ac_decomp *d = new (std::nothrow) ac_decomp();
    if (!d) return AC_ERR_OOM;
    d->grid = *grid;
    d->params = *params;
    for (int a = 0; a < 3; ++a) {
        d->p[a] = p[a];
        d->nloc[a] = nloc[a];
    }
    d->nsub = p[0] * p[1] * p[2];
    const double dx[3] = {grid->lx / grid->nx, grid->ly / grid->ny, grid->lz / grid->nz};
    d->coefs = make_coefs(dx, 3);
    d->phys = make_phys(*params);
    d->elem_f = params->precision == AC_FP64 ? 8 : 4;
    d->elem_w = params->precision == AC_FP32 ? 4 : 8;
    d->stream = static_cast<cudaStream_t>(stream);
    d->overlap = 1;
    const int rc = dc_setup(d);
    if (rc) {
        dc_free(d);
        delete d;
        return rc;
    }
    *out = d;
    return AC_OK;
}

extern "C" int ac_decomp_quit(ac_decomp *d) {
    if (!d) return AC_OK;
    cudaStreamSynchronize(d->stream);
    cudaStreamSynchronize(d->comm);
    dc_free(d);
    delete d;
    return AC_OK;
}

extern "C" int ac_decomp_set_overlap(ac_decomp *d, int on) {
    if (!d) return AC_ERR_ARG;
    d->overlap = on != 0;
    return AC_OK;
}

extern "C" int ac_decomp_info(const ac_decomp *d, int p[3], int nloc[3], int *messages,
                              unsigned long long *launches) {
    if (!d) return AC_ERR_ARG;
    for (int a = 0; a < 3; ++a) {
        if (p) p[a] = d->p[a];
        if (nloc) nloc[a] = d->nloc[a];
    }
    if (messages) *messages = (int)d->msgs.size();
    if (launches) *launches = d->launches;
    return AC_OK;
}

// Host float64 global array <-> the subdomains' interiors (binary64 staging of
// one subdomain at a time; synchronous).
static int dc_transfer(ac_decomp *d, int field, double *host, int to_dev, int to_w) {
    if (!d || !host || field < AC_ALL || field >= NF) return AC_ERR_ARG;
    const int q0 = field == AC_ALL ? 0 : field, q1 = field == AC_ALL ? NF : field + 1;
    const size_t n = (size_t)d->grid.nx * d->grid.ny * d->grid.nz;
    std::vector<double> tmp(d->stage_elems);
    const Geom lg = make_geom(d->nloc[0], d->nloc[1], d->nloc[2], AC_LAYOUT_PADDED);
    for (int q = q0; q < q1; ++q) {
        double *h = host + (field == AC_ALL ? (size_t)q * n : 0);
        for (int r = 0; r < d->nsub; ++r) {
            DcSub &s = d->sub[r];
            void *arr = to_w ? s.w[q] : s.state[d->cur][q];
            const int es = to_w ? d->elem_w : d->elem_f;
            if (!to_dev) {
                DCK(launch_gather(arr, es, lg, 0, d->nloc[2], d->stage, d->stream));
                d->launches++;
                DCK(cudaMemcpyAsync(tmp.data(), d->stage, d->stage_elems * sizeof(double),
                                    cudaMemcpyDeviceToHost, d->stream));
                DCK(cudaStreamSynchronize(d->stream));
            }
            for (int k = 0; k < d->nloc[2]; ++k)
                for (int j = 0; j < d->nloc[1]; ++j) {
                    double *row = h + ((size_t)(s.off[2] + k) * d->grid.ny + s.off[1] + j) *
                                          d->grid.nx + s.off[0];
                    double *loc = tmp.data() + ((size_t)k * d->nloc[1] + j) * d->nloc[0];
                    if (to_dev)
                        memcpy(loc, row, d->nloc[0] * sizeof(double));
                    else
                        memcpy(row, loc, d->nloc[0] * sizeof(double));
                }
            if (to_dev) {
                DCK(cudaMemcpyAsync(d->stage, tmp.data(), d->stage_elems * sizeof(double),
                                    cudaMemcpyHostToDevice, d->stream));
                DCK(launch_scatter(d->stage, arr, es, lg, 0, d->nloc[2], d->stream));
                d->launches++;
                DCK(cudaStreamSynchronize(d->stream));
            }
        }
    }
    if (to_dev && !to_w) d->next_s = 0;
    return AC_OK;
}

extern "C" int ac_decomp_load(ac_decomp *d, int field, const double *host_src) {
    return dc_transfer(d, field, const_cast<double *>(host_src), 1, 0);
}
extern "C" int ac_decomp_store(ac_decomp *d, int field, double *host_dst) {
    return dc_transfer(d, field, host_dst, 0, 0);
}
extern "C" int ac_decomp_load_w(ac_decomp *d, int field, const double *host_src) {
    return dc_transfer(d, field, const_cast<double *>(host_src), 1, 1);
}
extern "C" int ac_decomp_store_w(ac_decomp *d, int field, double *host_dst) {
    return dc_transfer(d, field, host_dst, 0, 1);
}

extern "C" int ac_decomp_integrate_substep(ac_decomp *d, double dt, int s) {
    AC_RANGE("ac_decomp_integrate_substep");
    if (!d || s < 0 || s > 2 || !isfinite(dt)) return AC_ERR_ARG;
    if (s != d->next_s) return AC_ERR_STATE;
    static const double alpha[3] = {0.0, -5.0 / 9.0, -153.0 / 128.0};
    static const double beta[3] = {1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0};
    if (d->params.force_amp != 0.0 && (!d->ftab_valid || d->ftab_step != d->step)) {
        ac_forcing_draw(d->params.seed, d->step, d->force_k, d->force_e, &d->force_phi);
        for (int r = 0; r < d->nsub; ++r) {
            const DcSub &sb = d->sub[r];
            const int total = sb.g.nx + sb.g.ny + sb.g.nz;
            dc_forcing_table_kernel<<<(total + 255) / 256, 256, 0, d->stream>>>(
                sb.g.nx, sb.g.ny, sb.g.nz, sb.off[0], sb.off[1], sb.off[2], d->grid.nx,
                d->grid.ny, d->grid.nz, d->force_k[0], d->force_k[1], d->force_k[2],
                cos(d->force_phi), sin(d->force_phi), sb.ftab);
            d->launches++;
        }
        DCK(cudaGetLastError());
        d->ftab_step = d->step;
        d->ftab_valid = 1;
    }
    const Geom *geoms = dc_geoms_dev(d);
    const int *nl = d->nloc;
    // update boxes in interior coordinates [0, n'): the whole interior, the inner
    // segment [r, n' - r) (its stencils read no halo cell) and the six slabs of
    // the outer segment
    const Box whole = {{0, 0, 0}, {nl[0], nl[1], nl[2]}};
    const Box inner = {{R, R, R}, {nl[0] - R, nl[1] - R, nl[2] - R}};
    Box outer[6];
    outer[0] = {{0, 0, 0}, {nl[0], nl[1], R}};                               // z low
    outer[1] = {{0, 0, nl[2] - R}, {nl[0], nl[1], nl[2]}};                   // z high
    outer[2] = {{0, 0, R}, {nl[0], R, nl[2] - R}};                           // y low
    outer[3] = {{0, nl[1] - R, R}, {nl[0], nl[1], nl[2] - R}};               // y high
    outer[4] = {{0, R, R}, {R, nl[1] - R, nl[2] - R}};                       // x low
    outer[5] = {{nl[0] - R, R, R}, {nl[0], nl[1] - R, nl[2] - R}};           // x high
    const long long nmsg = d->msg_elems;
    const unsigned dblocks = (unsigned)(((nmsg + 255) / 256) < 152 * 8 ? (nmsg + 255) / 256 : 152 * 8);
    if (d->overlap) {
        // the comm stream starts after everything queued so far (previous substep)
        DCK(cudaEventRecord(d->ev_start, d->stream));
        DCK(cudaStreamWaitEvent(d->comm, d->ev_start, 0));
        DCK(ac::dc_pack<true>(d, d->sendbuf, d->comm, geoms));
        if (d->elem_f == 8)
            dc_deliver_kernel<double><<<dblocks, 256, 0, d->comm>>>(
                static_cast<const double *>(d->sendbuf), static_cast<double *>(d->recvbuf), nmsg);
        else
            dc_deliver_kernel<float><<<dblocks, 256, 0, d->comm>>>(
                static_cast<const float *>(d->sendbuf), static_cast<float *>(d->recvbuf), nmsg);
        d->launches++;
        DCK(cudaGetLastError());
        DCK(ac::dc_pack<false>(d, d->recvbuf, d->comm, geoms));
        DCK(cudaEventRecord(d->ev_unpacked, d->comm));
        // the inner segments read no halo cell: they run while the halos are exchanged
        for (int r = 0; r < d->nsub; ++r)
            DCK(ac::dc_update(d, r, inner, alpha[s], beta[s], dt, s, d->stream));
        // the outer slabs start once the halos are in (the unpack event follows the
        // previous substep and this step's forcing tables through the comm stream),
        // alongside the inner updates, spread over the outer streams and joined back
        for (int k = 0; k < ac_decomp::DC_OUTER; ++k)
            DCK(cudaStreamWaitEvent(d->outer[k], d->ev_unpacked, 0));
        int job = 0;
        for (int r = 0; r < d->nsub; ++r)
            for (int b = 0; b < 6; ++b, ++job)
                DCK(ac::dc_update(d, r, outer[b], alpha[s], beta[s], dt, s,
                                  d->outer[job % ac_decomp::DC_OUTER]));
        for (int k = 0; k < ac_decomp::DC_OUTER; ++k) {
            DCK(cudaEventRecord(d->ev_outer[k], d->outer[k]));
            DCK(cudaStreamWaitEvent(d->stream, d->ev_outer[k], 0));
        }
    } else {
        DCK(ac::dc_pack<true>(d, d->sendbuf, d->stream, geoms));
        if (d->elem_f == 8)
            dc_deliver_kernel<double><<<dblocks, 256, 0, d->stream>>>(
                static_cast<const double *>(d->sendbuf), static_cast<double *>(d->recvbuf), nmsg);
        else
            dc_deliver_kernel<float><<<dblocks, 256, 0, d->stream>>>(
                static_cast<const float *>(d->sendbuf), static_cast<float *>(d->recvbuf), nmsg);
        d->launches++;
        DCK(cudaGetLastError());
        DCK(ac::dc_pack<false>(d, d->recvbuf, d->stream, geoms));
        for (int r = 0; r < d->nsub; ++r)
            DCK(ac::dc_update(d, r, whole, alpha[s], beta[s], dt, s, d->stream));
    }
    d->cur = 1 - d->cur;
    d->next_s = (s + 1) % 3;
    if (s == 2) d->step++;
    return AC_OK;
}

extern "C" int ac_decomp_integrate_step(ac_decomp *d, double dt) {
    if (!d || !isfinite(dt)) return AC_ERR_ARG;
    if (d->next_s != 0) return AC_ERR_STATE;
    for (int s = 0; s < 3; ++s) {
        const int rc = ac_decomp_integrate_substep(d, dt, s);
        if (rc) return rc;
    }
    return AC_OK;
}

AC_BC_READER(bc_take_decomp)
