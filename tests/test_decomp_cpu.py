"""Host logic of the domain decomposition (Sec. 3.2-3.3), no GPU:

  * the partition of a power-of-two device count, P = morton^-1(C_P - 1) + (1, 1, 1),
    against the bit interleaving the paper spells out (abcdef_2 -> (cf_2, be_2, ad_2));
  * the Z-order mapping of ranks to subdomain coordinates (a permutation; on a
    power-of-two cube it is morton^-1 itself);
  * the halo-segment schedule the library uses (ac_decomp_segment): every side
    and edge of every subdomain, exchanged between two gloo ranks (and between
    eight subdomains in one process) as the messages of Sec. 3.3, must leave
    each halo equal to the periodic images np.pad(mode="wrap") gives, corners
    aside (the Eq. 13 stencil never reads them).
"""
import itertools
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
R = 3


@pytest.fixture(scope="module")
def ac():
    from paper_2103_01597_gb300 import ac as _ac, build
    build.build()
    _ac.load_library()
    return _ac


def morton_inverse(i):
    """(x, y, z) of a Z-order index: bit 3b of i is bit b of x, 3b+1 of y, 3b+2 of z."""
    c = [0, 0, 0]
    for b in range(11):
        for a in range(3):
            c[a] |= ((i >> (3 * b + a)) & 1) << b
    return tuple(c)


def test_morton_inverse_matches_the_papers_example():
    # abcdef_2 -> (cf_2, be_2, ad_2): a = bit 5 ... f = bit 0
    for i in range(64):
        a, b, c, d, e, f = [(i >> k) & 1 for k in (5, 4, 3, 2, 1, 0)]
        assert morton_inverse(i) == (2 * c + f, 2 * b + e, 2 * a + d)


def test_partition_of_power_of_two_counts(ac):
    for k in range(10):
        count = 1 << k
        p = ac.ac_decomp_partition(count)
        assert p == tuple(v + 1 for v in morton_inverse(count - 1))
        assert p[0] * p[1] * p[2] == count
    assert ac.ac_decomp_partition(8) == (2, 2, 2)
    assert ac.ac_decomp_partition(2) == (2, 1, 1)
    for bad in (0, 3, 6, 1024):
        with pytest.raises(ac.AcError):
            ac.ac_decomp_partition(bad)


def test_zorder_rank_mapping(ac):
    for p in [(2, 2, 2), (4, 4, 4), (2, 1, 1), (1, 1, 8), (3, 2, 5)]:
        coords = [ac.ac_decomp_coord(p, r) for r in range(p[0] * p[1] * p[2])]
        assert sorted(coords) == sorted(itertools.product(*[range(v) for v in p]))
    for r in range(64):
        assert ac.ac_decomp_coord((4, 4, 4), r) == morton_inverse(r)


def _segments(ac, nloc):
    segs = [ac.ac_decomp_segment(nloc, k) for k in range(18)]
    dirs = [s[0] for s in segs]
    assert len(set(dirs)) == 18
    assert all(1 <= sum(abs(v) for v in d) <= 2 for d in dirs)  # sides and edges only
    return segs


def _box(a, b0, ext):
    return a[..., b0[2]:b0[2] + ext[2], b0[1]:b0[1] + ext[1], b0[0]:b0[0] + ext[0]]


def _expected(glob, coord, nloc):
    """The subdomain's padded window of the periodically padded global field."""
    pad = np.pad(glob, R, mode="wrap")
    o = [c * n for c, n in zip(coord, nloc)]
    return pad[o[2]:o[2] + nloc[2] + 2 * R, o[1]:o[1] + nloc[1] + 2 * R,
               o[0]:o[0] + nloc[0] + 2 * R]


def _no_corner_mask(nloc):
    m = np.ones(tuple(v + 2 * R for v in nloc[::-1]), dtype=bool)
    outside = [np.zeros(v + 2 * R, dtype=bool) for v in nloc[::-1]]
    for o, v in zip(outside, nloc[::-1]):
        o[:R] = True
        o[R + v:] = True
    zz, yy, xx = np.meshgrid(*outside, indexing="ij")
    m &= (zz.astype(int) + yy + xx) < 3
    return m


def test_schedule_fills_halos_in_one_process(ac):
    """Eight subdomains (2 x 2 x 2) and a 1 x 3 x 2 split exchanging all their
    messages in one process."""
    rng = np.random.default_rng(3)
    for n, p in [((16, 12, 20), (2, 2, 2)), ((7, 18, 12), (1, 3, 2))]:
        glob = rng.standard_normal(n[::-1])
        nloc = tuple(a // b for a, b in zip(n, p))
        segs = _segments(ac, nloc)
        ranks = p[0] * p[1] * p[2]
        coord = [ac.ac_decomp_coord(p, r) for r in range(ranks)]
        rank_of = {c: r for r, c in enumerate(coord)}
        loc = []
        for r in range(ranks):
            a = np.zeros(tuple(v + 2 * R for v in nloc[::-1]))
            o = [c * m for c, m in zip(coord[r], nloc)]
            a[R:R + nloc[2], R:R + nloc[1], R:R + nloc[0]] = \
                glob[o[2]:o[2] + nloc[2], o[1]:o[1] + nloc[1], o[0]:o[0] + nloc[0]]
            loc.append(a)
        for r in range(ranks):  # receiver r, segment k: sent by the neighbour at +d
            for d, src, dst, ext in segs:
                sender = rank_of[tuple((c + v) % m for c, v, m in zip(coord[r], d, p))]
                _box(loc[r], dst, ext)[...] = _box(loc[sender], src, ext)
        mask = _no_corner_mask(nloc)
        for r in range(ranks):
            want = _expected(glob, coord[r], nloc)
            assert np.array_equal(loc[r][mask], want[mask]), (n, p, r)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    from paper_2103_01597_gb300 import ac
    ac.load_library()
    dist.init_process_group("gloo", rank=rank, world_size=2)
    try:
        n, p = (12, 10, 8), (2, 1, 1)
        nloc = tuple(a // b for a, b in zip(n, p))
        glob = np.random.default_rng(5).standard_normal(n[::-1])  # the same on both ranks
        coord = ac.ac_decomp_coord(p, rank)
        rank_of = {ac.ac_decomp_coord(p, r): r for r in range(2)}
        a = np.zeros(tuple(v + 2 * R for v in nloc[::-1]))
        o = [c * m for c, m in zip(coord, nloc)]
        a[R:R + nloc[2], R:R + nloc[1], R:R + nloc[0]] = \
            glob[o[2]:o[2] + nloc[2], o[1]:o[1] + nloc[1], o[0]:o[0] + nloc[0]]
        interior = a.copy()
        reqs, inbox = [], []
        for k in range(18):  # the halo exchange: isend every outbound, irecv every inbound
            d, src, dst, ext = ac.ac_decomp_segment(nloc, k)
            recv_from = rank_of[tuple((c + v) % m for c, v, m in zip(coord, d, p))]
            send_to = rank_of[tuple((c - v) % m for c, v, m in zip(coord, d, p))]
            msg = torch.from_numpy(np.ascontiguousarray(_box(interior, src, ext)))
            buf = torch.empty_like(msg)
            if send_to == rank and recv_from == rank:
                buf.copy_(msg)
            else:
                reqs.append(dist.isend(msg, send_to, tag=k))
                reqs.append(dist.irecv(buf, recv_from, tag=k))
            inbox.append((dst, ext, buf))
        for q in reqs:
            q.wait()
        for dst, ext, buf in inbox:  # unpack
            _box(a, dst, ext)[...] = buf.numpy()
        mask = _no_corner_mask(nloc)
        want = _expected(glob, coord, nloc)
        out.put((rank, bool(np.array_equal(a[mask], want[mask]))))
    finally:
        dist.destroy_process_group()


def test_schedule_exchange_between_two_gloo_ranks(ac):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    assert got == [(0, True), (1, True)]
