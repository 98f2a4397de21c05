"""Pins for the oracle MLP: backpropagation against central finite differences."""
import numpy as np

from oracle import mlp


def test_mlp_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    sizes = [7, 6, 5, 4]
    Ws = [rng.standard_normal((sizes[i + 1], sizes[i])) * 0.5 for i in range(3)]
    bs = [rng.standard_normal(sizes[i + 1]) * 0.1 for i in range(3)]
    x = rng.standard_normal((9, sizes[0]))
    y = rng.standard_normal((9, sizes[-1]))
    mask = (rng.uniform(size=y.shape) > 0.3).astype(float)
    L, dWs, dbs = mlp.backward(x, Ws, bs, y, mask)
    h = 1e-6
    for l in range(3):
        for (i, j) in [(0, 0), (1, 2), (sizes[l + 1] - 1, sizes[l] - 1)]:
            Wp = [W.copy() for W in Ws]
            Wm = [W.copy() for W in Ws]
            Wp[l][i, j] += h
            Wm[l][i, j] -= h
            fd = (mlp.loss(mlp.forward(x, Wp, bs)[0], y, mask) - mlp.loss(mlp.forward(x, Wm, bs)[0], y, mask)) / (2 * h)
            assert abs(fd - dWs[l][i, j]) < 1e-6 * (1 + abs(fd))
        bp = [b.copy() for b in bs]
        bm = [b.copy() for b in bs]
        bp[l][0] += h
        bm[l][0] -= h
        fd = (mlp.loss(mlp.forward(x, Ws, bp)[0], y, mask) - mlp.loss(mlp.forward(x, Ws, bm)[0], y, mask)) / (2 * h)
        assert abs(fd - dbs[l][0]) < 1e-6 * (1 + abs(fd))
    # ReLU layers pass zero gradient where the pre-activation is negative; loss is 0 at the target
    out = mlp.forward(x, Ws, bs)[0]
    assert mlp.loss(out, out, mask) == 0.0
