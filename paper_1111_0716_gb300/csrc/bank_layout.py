"""Shared-memory bank-conflict model of the plane transforms in xx_kernels.cuh.

The plane transforms (plane_forward, plane_inverse) exchange data through a
shared buffer of N rows of LD complex values. Between the two steps of the x
transform, row y holds slot k1*S + n2. This script counts, for the kernels'
thread mappings, how many shared-memory wavefronts those accesses take. It
chose the slot stride S and row length LD of each grid length (the Lay<N>
table), and the tests use it to check the table.

Model. Shared memory has 32 banks of 4 bytes. A warp's 8-byte accesses (FP32
complex) are served in two half-warp phases of 16 lanes, 128 bytes each.
Element e lies in bank pair e mod 16. A phase costs as many wavefronts as the
largest number of distinct elements that share one bank pair (lanes reading
the same element share its wavefront). The ideal is one wavefront per phase
that has an active lane. A buffer's base offset shifts every address by the
same amount, so it does not change the count.

Run from this directory:
    python bank_layout.py            # ratios of the committed layouts
    python bank_layout.py --search   # best (S, LD) per N over the search space
"""
import math
import os
import re
import sys

HERE = os.path.dirname(os.path.abspath(__file__))


def lay_from_header(path=os.path.join(HERE, "xx_kernels.cuh")):
    """{N: (A, B, S, LD)} from the Lay<N> specialisations."""
    src = open(path).read()
    pat = (r"template <> struct Lay<(\d+)> \{ static constexpr int A = (\d+), B = (\d+), "
           r"S = (\d+), LD = (\d+); \};")
    return {int(m[0]): tuple(int(v) for v in m[1:]) for m in re.findall(pat, src)}


def round_up(x, m):
    return (x + m - 1) // m * m


def lcm(a, b):
    return a * b // math.gcd(a, b)


def nt_one_buffer(N, A, B):
    """Threads of a one-buffer plane (pass A, FP64 planes): PlaneCfg's default."""
    return round_up(N * A // 2, lcm(lcm(32, B), 1 if A == 8 else A))


def nt_two_buffers(N, A):
    """Threads of a two-buffer plane (FP32 pass C)."""
    return round_up(N * A, 32)


def nt_staged(N, A, B):
    """Threads of the staged pass A (one buffer, one item per thread)."""
    return round_up(N * A, lcm(lcm(32, B), 1 if A == 8 else A))


def x2_item(A, it):
    """(k1, row) of second-x-step item it (the kernel's x2_item)."""
    if A == 8:
        lane, warp = it & 31, it >> 5
        return (lane & 3) | ((lane >> 4) << 2), 4 * warp + ((lane >> 2) & 3)
    return it % A, it // A


def phase_cost(addrs):
    """(wavefronts, ideal) of one warp access; addrs: 32 element indices or None."""
    cost = ideal = 0
    for half in (addrs[:16], addrs[16:]):
        banks = {}
        for a in half:
            if a is not None:
                banks.setdefault(a % 16, set()).add(a)
        if banks:
            cost += max(len(v) for v in banks.values())
            ideal += 1
    return cost, ideal


def _sum(costs):
    c = i = 0
    for a, b in costs:
        c += a
        i += b
    return c, i


def _warps(NT, n_items):
    """Lists of 32 item indices (None past n_items), one per warp instruction."""
    for i in range((n_items + NT - 1) // NT):
        for w in range(NT // 32):
            yield [w * 32 + l + i * NT if w * 32 + l + i * NT < n_items else None
                   for l in range(32)]


def x_forward(N, A, B, S, LD, NT):
    """x transform of plane_forward: step 1 stores slots, step 2 loads slots and
    stores natural positions."""
    out = []
    for its in _warps(NT, N * B):
        for k1 in range(A):
            out.append(phase_cost([None if it is None else (it // B) * LD + k1 * S + it % B
                                   for it in its]))
    for its in _warps(NT, N * A):
        kr = [None if it is None else x2_item(A, it) for it in its]
        for n2 in range(B):
            out.append(phase_cost([None if x is None else x[1] * LD + x[0] * S + n2 for x in kr]))
        for k2 in range(B):
            out.append(phase_cost([None if x is None else x[1] * LD + x[0] + A * k2 for x in kr]))
    return _sum(out)


def x_inverse(N, A, B, S, LD, NT):
    """x transform of plane_inverse (every input column counted, as unpruned):
    step 1 loads natural positions and stores slots, step 2 loads slots."""
    out = []
    for its in _warps(NT, N * B):
        for n1 in range(A):
            out.append(phase_cost([None if it is None else (it // B) * LD + B * n1 + it % B
                                   for it in its]))
        for k1 in range(A):
            out.append(phase_cost([None if it is None else (it // B) * LD + k1 * S + it % B
                                   for it in its]))
    for its in _warps(NT, N * A):
        kr = [None if it is None else x2_item(A, it) for it in its]
        for n2 in range(B):
            out.append(phase_cost([None if x is None else x[1] * LD + x[0] * S + n2 for x in kr]))
    return _sum(out)


def x_cost(N, A, B, S, LD):
    """The searched objective: a one-buffer forward plus a two-buffer inverse."""
    f = x_forward(N, A, B, S, LD, nt_one_buffer(N, A, B))
    i = x_inverse(N, A, B, S, LD, nt_two_buffers(N, A))
    return f[0] + i[0], f[1] + i[1]


def y_columns(N, h):
    """Columns (natural f_x index) of kept column kxb < 2h + 1 (the kernel's
    idx_of_box): -h..-1 at N - h..N - 1, then 0..h."""
    return [kxb - h if kxb >= h else kxb - h + N for kxb in range(2 * h + 1)]


def y_cost(N, h):
    """(wavefronts, ideal) per warp-instruction pair of the y steps over kept
    columns, lanes over consecutive kxb: every y-step access of a warp has
    the same row for all lanes, so only the columns decide conflicts."""
    cols = y_columns(N, h)
    cost = ideal = 0
    for cb in range(0, len(cols), 32):
        lanes = cols[cb:cb + 32]
        c, i = phase_cost(lanes + [None] * (32 - len(lanes)))
        cost += c
        ideal += i
    return cost, ideal


def staged_read_cost(N, A, B, pitch=None):
    """(wavefronts, ideal) of the staged pass A's first x step reading the
    bulk-copied occupied plane (row pitch N as committed, or `pitch`): lane item
    it reads row it / B, column B*n1 + it % B."""
    pitch = N if pitch is None else pitch
    out = []
    for its in _warps(nt_staged(N, A, B), N * B):
        for n1 in range(A):
            out.append(phase_cost([None if it is None else (it // B) * pitch + B * n1 + it % B
                                   for it in its]))
    return _sum(out)


def conflict_free_pitch(N, B):
    """Smallest row pitch >= N equal to B modulo 16: lane item it then reads element
    it + B*n1 (mod 16), so a half-warp hits 16 distinct bank pairs."""
    pitch = N
    while pitch % 16 != B % 16:
        pitch += 1
    return pitch


def search(N, A, B):
    """[(wavefronts, S, LD)] over S in [B, B + 16], LD in [max(N, (A-1) S + B), N + 40],
    sorted."""
    res = []
    for S in range(B, B + 17):
        for LD in range(max(N, (A - 1) * S + B), N + 41):
            res.append((x_cost(N, A, B, S, LD)[0], S, LD))
    res.sort()
    return res


def main(argv):
    lay = lay_from_header()
    for N, (A, B, S, LD) in sorted(lay.items()):
        c, i = x_cost(N, A, B, S, LD)
        line = "N=%2d S=%2d LD=%3d  x steps %.3f" % (N, S, LD, c / i)
        h = 2 * ((N - 1) // 4)                # widest kept half-width 2 n_max, 4 n_max + 1 <= N
        yc, yi = y_cost(N, h)
        sc, si = staged_read_cost(N, A, B)
        line += "  y steps (h=%d) %.3f  staged reads %.3f" % (h, yc / yi, sc / si)
        if "--search" in argv:
            best = search(N, A, B)[0]
            line += "  best %d at S=%d LD=%d (committed %d)" % (best[0], best[1], best[2], c)
        print(line)


if __name__ == "__main__":
    main(sys.argv[1:])
