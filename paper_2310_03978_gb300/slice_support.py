"""Which slices of a sliced network can contribute (host logic, no GPU, no contraction).

With fSim at theta = pi/2 and no final single-qubit layer, the gate swaps its two wires (times
phases), so a closed qubit's projector after its last fSim fixes the partner's input bond; when
that bond is sliced, only the matching slices contribute and the others are exactly zero.  To
compare precisions on slices that carry amplitude, ``supported_slices`` draws slice ids that no
tensor forces to zero: ``slice_constraints`` lists, per tensor (alone, and for a gate with its
neighbouring vectors absorbed), the value tuples of its sliced bonds on which it is not
identically zero.  These conditions are necessary, not sufficient.
"""
from __future__ import annotations

import numpy as np


def slice_constraints(net, sliced):
    """Necessary conditions for a slice to contribute: for every tensor, alone and (for a gate)
    with its neighbouring vectors (|0> inputs, <b| projectors) absorbed, the value tuples of its
    sliced bonds on which it is not identically zero (entries below 1e-12 of its largest count as
    zero).  Returns [(bit positions in the slice id, allowed value tuples)] for the tensors that
    exclude some tuple.  A projector after a swap-like fSim fixes the partner's input bond."""
    import itertools
    pos = {l: j for j, l in enumerate(sliced)}
    vec = {ls[0]: t for t, ls in zip(net.tensors, net.labels) if len(ls) == 1}
    pieces = list(zip(net.tensors, net.labels))
    for t, ls in zip(net.tensors, net.labels):
        if len(ls) < 2 or not any(l in vec for l in ls):
            continue
        ls = list(ls)
        for l in list(ls):
            if l in vec:
                t = np.tensordot(t, vec[l], axes=([ls.index(l)], [0]))
                ls.remove(l)
        pieces.append((t, ls))
    cons = []
    for t, ls in pieces:
        axes = [i for i, l in enumerate(ls) if l in pos]
        if not axes:
            continue
        big = np.abs(t) > 1e-12 * np.abs(t).max()
        ok = set()
        for vals in itertools.product((0, 1), repeat=len(axes)):
            idx = [slice(None)] * t.ndim
            for a, v in zip(axes, vals):
                idx[a] = v
            if big[tuple(idx)].any():
                ok.add(vals)
        if len(ok) < 1 << len(axes):
            cons.append(([pos[ls[a]] for a in axes], ok))
    return cons


def slice_supported(cons, s):
    """Whether slice id ``s`` meets every condition of ``slice_constraints``."""
    return all(tuple((s >> b) & 1 for b in bits) in ok for bits, ok in cons)


def supported_slices(net, sliced, seed, count):
    """Up to ``count`` distinct slice ids (bit j = value of sliced[j]) that meet
    ``slice_constraints``: a seeded depth-first search over the bits with the values tried in
    random order."""
    cons = slice_constraints(net, sliced)
    by_bit = [[] for _ in sliced]
    for c in cons:
        for b in c[0]:
            by_bit[b].append(c)
    rng = np.random.default_rng(seed)
    found = []
    for _ in range(64 * count):
        if len(found) == count:
            break
        val = [-1] * len(sliced)

        def fits(b):
            for bits, ok in by_bit[b]:
                if not any(all(val[x] < 0 or val[x] == v for x, v in zip(bits, vs)) for vs in ok):
                    return False
            return True

        def dfs(b):
            if b == len(sliced):
                return True
            for v in rng.permutation(2):
                val[b] = int(v)
                if fits(b) and dfs(b + 1):
                    return True
            val[b] = -1
            return False

        if dfs(0):
            s = sum(v << j for j, v in enumerate(val))
            if s not in found:
                found.append(s)
    return found
