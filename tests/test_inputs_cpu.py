"""The seeded workload generators: reproducible, and within the recipe's bounds
(separation, margin, counts, coupling ranges). CPU only."""
import itertools
import math

from paper_2603_24370_gb300 import inputs as I


def test_generators_are_reproducible():
    assert [p.solitons for p in I.ah_batch(5, 3)] == [p.solitons for p in I.ah_batch(5, 3)]
    assert [p.solitons for p in I.cm_learned_set(5, 3)] == [p.solitons for p in I.cm_learned_set(5, 3)]


def test_ah_batch_recipe():
    for p in I.ah_batch(64):
        L = p.nx * p.dx
        assert p.nx in (64, 128, 256, 512) and p.nx == p.ny and p.dx == 0.1
        assert 0.5 <= p.params[0] < 2.0 and 1 <= len(p.solitons) <= 4
        assert all(abs(s[0]) <= L / 4 and abs(s[1]) <= L / 4 for s in p.solitons)


def test_chiral_magnet_sets_keep_separation_and_margin():
    for p in I.cm_learned_set(32, side=256) + [I.cm_skyrmions(n=1024)]:
        half = 0.5 * (p.nx - 1) * p.dx
        assert 1 <= len(p.solitons) <= max(4, 8)
        for a, b in itertools.combinations(p.solitons, 2):
            assert math.hypot(a[0] - b[0], a[1] - b[1]) >= 8.0
        assert all(abs(s[0]) <= half - 8.0 and abs(s[1]) <= half - 8.0 for s in p.solitons)
        assert all(s[2] == 1.0 and s[3] == 2.0 for s in p.solitons)
