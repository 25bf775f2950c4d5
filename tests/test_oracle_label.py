"""Droplet labelling of the oracle against an independent brute-force union-find.

Rule: components of {psi > 0} over fluid sites, face-connected, periodic axes
wrap; each component is labelled by its smallest linear site index, -1 elsewhere."""
import itertools

import numpy as np
import pytest

import oracle
from paper_1711_02003_gb300 import workloads as W


def brute_labels(dims, periodic, field):
    n = int(np.prod(dims))
    parent = list(range(n))

    def find(a):
        while parent[a] != a:
            a = parent[a]
        return a
    strides = [1]
    for d in dims[:-1]:
        strides.append(strides[-1] * d)
    for s in range(n):
        if not field[s]:
            continue
        coord = [(s // strides[a]) % dims[a] for a in range(len(dims))]
        for a in range(len(dims)):
            c2 = list(coord)
            c2[a] += 1
            if c2[a] == dims[a]:
                if not periodic[a]:
                    continue
                c2[a] = 0
            t = sum(c2[b] * strides[b] for b in range(len(dims)))
            if field[t]:
                ra, rb = find(s), find(t)
                if ra != rb:
                    parent[max(ra, rb)] = min(ra, rb)
    out = np.full(n, -1, np.int32)
    for s in range(n):
        if field[s]:
            # smallest index of the component
            out[s] = find(s)
    mins = {}
    for s in range(n):
        if field[s]:
            mins.setdefault(out[s], s)
    return np.array([mins[out[s]] if field[s] else -1 for s in range(n)], np.int32)


@pytest.mark.parametrize("dims", [(3, 3), (4, 4)])
@pytest.mark.parametrize("periodic", [(0, 0), (1, 1), (1, 0)])
def test_every_small_mask(dims, periodic):
    n = dims[0] * dims[1]
    step = 1 if n <= 9 else 7          # 4x4: every 7th of the 65536 masks (9363 masks)
    for bits in range(0, 1 << n, step):
        field = np.array([(bits >> s) & 1 for s in range(n)], np.uint8)
        assert np.array_equal(oracle.label_field(dims, periodic, field), brute_labels(dims, periodic, field))


def test_random_3d_fields():
    rng = np.random.default_rng(7)
    for _ in range(100):
        dims = tuple(int(v) for v in rng.integers(2, 6, 3))
        periodic = tuple(int(v) for v in rng.integers(0, 2, 3))
        field = (rng.random(int(np.prod(dims))) < 0.45).astype(np.uint8)
        assert np.array_equal(oracle.label_field(dims, periodic, field), brute_labels(dims, periodic, field))


def test_sim_label_two_droplets_across_periodic_edge():
    pb = W.static_droplet(W.D2Q9, 40, 5, centre=(0, 20, 0))
    # add a second droplet at (25, 8)
    y, x = np.mgrid[0:40, 0:40]
    second = ((x - 25) ** 2 + (y - 8) ** 2 < 16).ravel()
    rr = np.where(second, 1.0, pb.rho_r)
    rb = np.where(second, 0.0, pb.rho_b)
    s = oracle.Sim(pb.replace(rho_r=rr, rho_b=rb))
    labels, counts, vols, nd = s.label()
    assert nd == 2
    field = ((rr - rb) > 0).astype(np.uint8)
    assert np.array_equal(labels, brute_labels((40, 40), (1, 1), field))
    assert counts.sum() == field.sum()
    assert np.all(vols > 0)
