"""Checks of the seeded input generator (no method arithmetic involved)."""
import numpy as np
import pytest

import synth


def test_splitmix64_reference_stream():
    # splitmix64 with seed 1234567: first outputs of the published algorithm
    # (Steele, Lea, Flood 2014), computed by the definition in this test.
    def ref(seed, k):
        out, s = [], seed
        for _ in range(k):
            s = (s + 0x9E3779B97F4A7C15) % 2**64
            z = s
            z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) % 2**64
            z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) % 2**64
            out.append(z ^ (z >> 31))
        return out
    g = synth.SplitMix64(1234567)
    assert [g.next_u64() for _ in range(5)] == ref(1234567, 5)
    # first output for seed 0 is the well-known constant
    assert synth.SplitMix64(0).next_u64() == 0xE220A8397B1DCDAF


def test_q1_element_textbook():
    # bilinear square, Laplacian: (1/6)[4 -1 -1 -2; ...] in lexicographic corner order
    ke = synth.element_heat(2, h=0.37)
    ref = np.array([[4, -1, -1, -2], [-1, 4, -2, -1], [-1, -2, 4, -1], [-2, -1, -1, 4]]) / 6.0
    assert np.allclose(ke, ref, atol=1e-15)


def test_hex8_heat_element_scaling_and_kernel():
    k1 = synth.element_heat(3, 1.0)
    k2 = synth.element_heat(3, 0.25)
    assert np.allclose(k2, 0.25 * k1, atol=1e-15)           # K_e proportional to h in 3D
    assert np.allclose(k1 @ np.ones(8), 0, atol=1e-14)
    # textbook diagonal of the trilinear cube Laplacian: 1/3
    assert np.allclose(np.diag(k1), 1.0 / 3.0)


def test_hex8_elasticity_rigid_modes():
    ke = synth.element_elasticity(0.5)
    X = np.array([[l & 1, (l >> 1) & 1, (l >> 2) & 1] for l in range(8)], float) * 0.5
    R = np.zeros((24, 6))
    for l in range(8):
        x, y, z = X[l]
        R[3 * l:3 * l + 3, :3] = np.eye(3)
        R[3 * l:3 * l + 3, 3] = [-y, x, 0]
        R[3 * l:3 * l + 3, 4] = [0, -z, y]
        R[3 * l:3 * l + 3, 5] = [z, 0, -x]
    assert abs(ke @ R).max() < 1e-14
    assert np.linalg.matrix_rank(ke) == 18
    assert np.allclose(ke, ke.T)


def test_config1_shape():
    p = synth.make_config(1)
    sd = p.subdomains[0]
    assert (sd.n, sd.m) == (289, 64)
    assert np.all(np.diff(sd.Bt.indptr) == 1)
    assert np.all(sd.Bt.data == 1.0)
    assert abs(sd.K @ np.ones(sd.n)).max() < 1e-13


def test_config2_gluing_counts():
    p = synth.make_config(2)
    ms = np.array([s.m for s in p.subdomains])
    assert len(p.subdomains) == 64 and all(s.n == 4913 for s in p.subdomains)
    # non-redundant gluing of a 4^3 split of a 65^3 node grid:
    # plane nodes (2 owners) 1 multiplier, line nodes (4) 3, cross points (8) 7
    G, parts, k = 65, 4, 16
    inner = [g for g in range(G) if g % k == 0 and 0 < g < G - 1]
    n_on = lambda c: sum(1 for g in range(G) if (g in inner) == c)
    plane = 3 * len(inner) * n_on(False) ** 2
    line = 3 * len(inner) ** 2 * n_on(False)
    cross = len(inner) ** 3
    assert p.n_dual == plane * 1 + line * 3 + cross * 7 == 39807
    assert (ms.min(), ms.max()) == (817, 1634)
    # every multiplier appears in exactly two subdomains with opposite signs
    tally = np.zeros(p.n_dual)
    count = np.zeros(p.n_dual, int)
    for s in p.subdomains:
        np.add.at(tally, s.lambda_map, s.Bt.data)
        np.add.at(count, s.lambda_map, 1)
    assert np.all(count == 2) and np.all(tally == 0)


def test_lattice_gluing_small():
    p = synth.elasticity_cubes((2, 2, 1), 2, 3, seed=5)
    count = np.zeros(p.n_dual, int)
    for s in p.subdomains:
        np.add.at(count, s.lambda_map, 1)
        assert len(s.fixed) == 6
        # each column is a signed unit vector
        assert np.all(np.diff(s.Bt.indptr) == 1)
    assert np.all(count == 2)


def test_seed_determinism():
    a = synth.elasticity_cubes((2, 2, 2), 8, 16, seed=7)
    b = synth.elasticity_cubes((2, 2, 2), 8, 16, seed=7)
    assert [s.n for s in a.subdomains] == [s.n for s in b.subdomains]
    c = synth.elasticity_cubes((2, 2, 2), 8, 16, seed=8)
    assert [s.n for s in a.subdomains] != [s.n for s in c.subdomains]
