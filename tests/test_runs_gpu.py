"""The coordinate-run flags of 2-D packs (tile_runs_kernel) against their definition.

The fast sweeps evaluate a tile with the run variant only when, for every aligned group of 16 valid
points of the tile, one coordinate takes a single value; the flag (1 + that coordinate, else 0)
sits in the first entry of the pack's free component.  A wrong flag would send a tile without runs
through the shared-term evaluation, so the flags are read back from the device packs (a one-rank
sharded state exposes them) and compared with the definition computed here."""
import numpy as np
import pytest

import ot_inputs as I

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2609_33814_b300")

TQ, NCOMP, GROUP = 128, 5, 16


def _grid_xy(sx, sy):
    iy, ix = np.meshgrid(np.arange(sy), np.arange(sx), indexing="ij")
    return np.stack([ix.ravel(), iy.ravel()], axis=1).astype(np.float32)


def _expected_flags(pts):
    n = len(pts)
    tiles = (n + TQ - 1) // TQ
    out = np.zeros(tiles, np.float32)
    for t in range(tiles):
        same = [True, True]
        for g0 in range(t * TQ, min((t + 1) * TQ, n), GROUP):
            grp = pts[g0:min(g0 + GROUP, n)]
            for k in range(2):
                same[k] &= bool(np.all(grp[:, k] == grp[0, k]))
        out[t] = 2.0 if same[1] else (1.0 if same[0] else 0.0)
    return out


CASES = {
    "row_major_32": lambda rng: (_grid_xy(32, 32), _grid_xy(32, 32)),
    "col_major_16": lambda rng: (_grid_xy(16, 16)[:, ::-1].copy(), _grid_xy(16, 16)[:, ::-1].copy()),
    "shuffled_20": lambda rng: (_grid_xy(20, 20)[rng.permutation(400)], _grid_xy(20, 20)[rng.permutation(400)]),
    "mixed_24_16x17": lambda rng: (_grid_xy(24, 24), _grid_xy(16, 17)),
    "random_cloud": lambda rng: (I.random_cloud(300, 2, 5), I.random_cloud(500, 2, 6)),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_tile_run_flags_match_definition(case):
    x, y = CASES[case](np.random.default_rng(3))
    ctx = P.Context(0)
    S = P.ShardState(ctx, x, y, I.uniform_weights(len(x), 1), I.uniform_weights(len(y), 2), 0, 1,
                     cost_scale=1.0 / 2048.0, omega=1.0, eps0=1.0, lam=1.0, precision="mufu", cert_every=0)
    for side, pts in ((0, x), (1, y)):
        tiles = (len(pts) + TQ - 1) // TQ
        buf = S.pack_get(side)
        pack = np.frombuffer(buf[:tiles * NCOMP * TQ * 4].tobytes(), np.float32).reshape(tiles, NCOMP, TQ)
        np.testing.assert_array_equal(pack[:, NCOMP - 1, 0], _expected_flags(pts), err_msg=f"{case} side {side}")
    S.close()
    ctx.close()
