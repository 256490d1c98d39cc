"""Pins of the oracle's target-driven sampled tuner (Sec. VI-A and its
tuning table): the candidate sets the table lists, the uniform block sample,
and the vote -- on a field built so that one configuration clearly wins, the
tuner that sees the whole field and the one that sees a sample agree, and
the winner is the configuration whose byte counts are lowest at most
tolerances (recomputed here from the oracle's own refactors)."""
import numpy as np

import oracle
from oracle import tune as tn
from oracle.pipeline import Scheme


def _anisotropic(n=48, seed=4):
    """Smooth in axes 0 and 1, rough along axis 2 with a profile shared by
    every (i0, i1): the level-0 coefficients of slices normal to axis 2 are
    smooth in-slice, so decomposition along axis 2 should win."""
    rng = np.random.default_rng(seed)
    i0, i1, i2 = np.meshgrid(*[np.arange(n)] * 3, indexing="ij")
    g = np.sin(i0 / 7.0) * np.cos(i1 / 9.0) + 0.5 * np.sin((i0 + i1) / 11.0)
    h = rng.standard_normal(n)[None, None, :]
    return (g * (1.0 + 0.5 * h) + 0.2 * np.sin(i2 / 5.0)).astype(np.float32)


def test_candidate_sets_follow_the_tuning_table():
    eb3 = tn.candidates("eb", 3)
    ps3 = tn.candidates("psnr", 3)
    assert len(eb3) == (1 + 6) * 4 and len(ps3) == 6 * 4
    assert {c.interp for c in ps3} == {"region"}
    assert {c.encoding for c in eb3} == {"generic"} and {c.encoding for c in ps3} == {"negabinary"}
    assert {c.decomp_axis for c in eb3} == {-1, 0, 1, 2}
    orders = {c.order for c in eb3 if c.interp == "region"}
    assert len(orders) == 6 and all(sorted(o) == [0, 1, 2] for o in orders)
    assert len(tn.candidates("eb", 2)) == 3 and len(tn.candidates("psnr", 2)) == 2
    assert all(c.degree == "cubic" for c in eb3 + ps3)


def test_sample_blocks_are_uniform_and_about_one_percent():
    for shape in [(512, 512, 512), (256, 384, 384), (100, 500, 500), (1800, 3600), (48, 48, 48)]:
        origins, b = tn.sample_blocks(shape)
        n = int(np.prod(shape))
        assert len(origins) >= 1
        frac = len(origins) * int(np.prod(b)) / n
        assert frac <= 0.01 or len(origins) == 1
        for o in origins:
            assert all(0 <= oa and oa + ba <= s for oa, ba, s in zip(o, b, shape))
        assert len(set(origins)) == len(origins)            # no block twice
    origins, b = tn.sample_blocks((512, 512, 512))
    assert b == (64, 64, 64) and len(origins) == 4          # 0.78 %: a fifth block would pass 1 %


def test_sampled_tuner_agrees_with_the_full_field_tuner():
    X = _anisotropic()
    cands = [Scheme(mode="eb", interp="level", degree="cubic", decomp_axis=d, encoding="generic")
             for d in (-1, 0, 1, 2)]
    cands += [Scheme(mode="eb", interp="region", degree="cubic", order=(0, 1, 2), decomp_axis=d,
                     encoding="generic") for d in (-1, 2)]
    full, votes_f, table_f = tn.tune(X, "eb", fraction=1.0, edge=48, cands=cands)
    part, votes_s, table_s = tn.tune(X, "eb", fraction=0.3, edge=24, cands=cands)
    assert full == part == cands[3]                          # per-level, decomposition along axis 2
    assert votes_f[3] >= 5 and votes_s[3] >= 5
    # the vote follows the byte counts: recompute one tolerance directly
    R = float(X.max() - X.min())
    tab = []
    for c in cands:
        h = oracle.refactor(X, c)
        tab.append(tn.block_bytes(h, 1e-4 * R, False))
    assert [t[2] for t in table_f] == tab
    assert min(range(len(tab)), key=lambda i: (tab[i], i)) == 3


def test_psnr_mode_tunes_per_region_only():
    X = _anisotropic(40, 5)
    w, votes, table = tn.tune(X, "psnr", fraction=1.0, edge=40,
                              cands=[c for c in tn.candidates("psnr", 3) if c.order == (0, 1, 2)])
    assert w.interp == "region" and w.encoding == "negabinary" and w.decomp_axis == 2
    assert sum(votes) >= 5
