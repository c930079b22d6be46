"""The sampled-patch helpers used by the large-mesh GPU parity tests agree
with the oracle's own colour pass (dense assembled patch solves) on meshes
small enough for it: every patch of a colour, and the set of DoFs a colour
may touch, for the Dirichlet kernel (both residuals) and the full kernel."""
import numpy as np
import pytest

from oracle.mg import Level, smooth
from paper_2405_18982_gb300 import inputs
from patch_sampling import PatchOracle, colour_touch_mask, sample_vertices


@pytest.mark.parametrize("variant", ["consistent", "paper", "full"])
@pytest.mark.parametrize("case", [(2, 2, 8), (2, 3, 4), (3, 2, 4), (3, 1, 2)], ids=lambda c: f"d{c[0]}k{c[1]}N{c[2]}")
def test_patch_oracle_equals_colour_pass(case, variant):
    dim, k, N = case
    lev = Level(dim, k, N, variant=variant)
    b = inputs.normal(30, lev.ndof)
    x0 = inputs.normal(31, lev.ndof)
    po = PatchOracle(dim, k, N, variant)
    for c in range(2 ** dim):
        x1 = smooth(lev, x0, b, colours=[c])
        mask = colour_touch_mask(dim, k, N, c, full=variant == "full")
        # outside the colour's spaces nothing changes; inside, something may
        assert np.array_equal(x1[~mask], x0[~mask])
        union = np.zeros(lev.ndof, bool)
        par = [(c >> e) & 1 for e in range(dim)]
        verts = np.stack(np.meshgrid(*[np.arange(2 - p, N, 2) for p in par], indexing="ij"),
                         axis=-1).reshape(-1, dim)
        for v in verts:
            idx, u = po.update(tuple(int(t) for t in v), b, x0)
            assert np.abs(x1[idx] - x0[idx] - u).max() <= 1e-12 * max(np.abs(u).max(), 1.0)
            assert not union[idx].any()          # same-colour spaces are disjoint
            union[idx] = True
        assert np.array_equal(union, mask)


def test_sample_vertices_cover_the_ends():
    for dim, N in ((2, 16), (3, 8)):
        for c in range(2 ** dim):
            vs = sample_vertices(dim, N, c, 5, 12)
            for e in range(dim):
                p = (c >> e) & 1
                got = {v[e] for v in vs}
                assert (2 - p) in got and (N - 1 - (1 - p)) in got
                assert all(v[e] % 2 == p and 1 <= v[e] <= N - 1 for v in vs)
