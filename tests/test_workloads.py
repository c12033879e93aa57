"""The seeded input generators (`workloads/`), shared by the oracle and the
CUDA path:

* SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) against its published
  output sequence from state 0: stream 0 at positions 0, 1, 2, ... is that
  sequence, because the keyed state (2^32 seed + i + 1) times the golden gamma
  is the sequential state after i + 1 steps;
* uniform01: the top 53 bits scaled to [0, 1);
* the benchmark's channel tree: binary, exactly round(V M) solid elements, and
  one face-connected network that touches the heat-sink patch (the structure
  of the paper's optimised designs);
* the thresholded field: exactly round(V M) solid elements;
* every generator is a pure function of its seed.
"""
from collections import deque

import numpy as np

import workloads as W

# published SplitMix64 outputs from state 0
SPLITMIX64_FROM_ZERO = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_splitmix64_published_sequence():
    got = [int(v) for v in W.splitmix64(0, np.arange(3))]
    assert got == SPLITMIX64_FROM_ZERO


def test_uniform01_is_top_53_bits():
    u = W.uniform01(0, 3)
    assert u[0] == (SPLITMIX64_FROM_ZERO[0] >> 11) * 2.0 ** -53
    v = W.uniform01(9, 100000)
    assert v.min() >= 0.0 and v.max() < 1.0 and abs(v.mean() - 0.5) < 0.01


def _components(solid, N):
    """Face-connected components of the solid elements (BFS)."""
    lab = -np.ones(solid.size, dtype=np.int64)
    ncomp = 0
    for s in np.flatnonzero(solid):
        if lab[s] >= 0:
            continue
        lab[s] = ncomp
        q = deque([s])
        while q:
            e = q.popleft()
            x, y, z = e % N, (e // N) % N, e // (N * N)
            for dx, dy, dz in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
                a, b, c = x + dx, y + dy, z + dz
                if 0 <= a < N and 0 <= b < N and 0 <= c < N:
                    f = a + N * (b + N * c)
                    if solid[f] and lab[f] < 0:
                        lab[f] = ncomp
                        q.append(f)
        ncomp += 1
    return lab, ncomp


def test_channel_tree_binary_exact_volume_connected_to_the_sink():
    N = 32
    x = W.channel_tree_density(N, 3, 0.2)
    assert set(np.unique(x)) <= {0.0, 1.0}
    assert int(x.sum()) == int(np.floor(0.2 * N ** 3 + 0.5))
    lab, ncomp = _components(x > 0.5, N)
    assert ncomp == 1
    # the network reaches the bottom face inside the Dirichlet patch (|x - 1/2| <= 0.1)
    ex, ey = np.arange(N)[None, :], np.arange(N)[:, None]
    bottom = (x[: N * N].reshape(N, N) > 0.5)
    in_patch = (np.abs((ex + 0.5) / N - 0.5) <= 0.1) & (np.abs((ey + 0.5) / N - 0.5) <= 0.1)
    assert np.any(bottom & in_patch)


def test_threshold_field_exact_volume():
    N = 16
    x = W.smoothed_threshold_density(N, 1, 0.3)
    assert set(np.unique(x)) <= {0.0, 1.0}
    assert int(x.sum()) == int(np.floor(0.3 * N ** 3 + 0.5))


def test_generators_are_pure_functions_of_the_seed():
    np.testing.assert_array_equal(W.channel_tree_density(16, 5, 0.2), W.channel_tree_density(16, 5, 0.2))
    np.testing.assert_array_equal(W.uniform01(4, 1000), W.uniform01(4, 1000))
    assert not np.array_equal(W.uniform01(4, 1000), W.uniform01(5, 1000))
