"""Pins of the operation census behind the benchmark's algorithmic flop count
(oracle/flop_census.py, orc_census_step).

The census counts the operations a result needs in the oracle's own step
functions: no operation by a constant 0 or 1, identical operations once,
symmetric matrix results once (upper triangle).  Hand-derived counts of
covariance transports pin those rules; a repeated hit costs nothing (shared
work counted once); the stored per-unit counts must match a fresh census.
"""
import numpy as np
import pytest

import oracle

RNG = np.random.default_rng(5)


def _c21():
    return RNG.uniform(0.1, 1.0, 21)


def test_identity_transport_costs_nothing():
    assert oracle.census_transport(np.eye(6), _c21()).tolist() == [0, 0, 0, 0]


def test_one_off_diagonal_entry():
    # J = I + a e0 e1^T: row 0 of J C is C_0k + a C_1k (6 multiplies, 6 adds);
    # of the upper triangle of J C J^T only (0,0) needs more: + a (JC)_01.
    J = np.eye(6)
    J[0, 1] = 0.7
    assert oracle.census_transport(J, _c21()).tolist() == [7, 7, 0, 0]


def test_dense_transport_counts_the_upper_triangle_once():
    # J C: 36 dot products of length 6 (6 multiplies, 5 adds each); the
    # result's 21 upper entries: 21 more such dot products.
    J = RNG.uniform(0.2, 2.0, (6, 6))
    assert oracle.census_transport(J, _c21()).tolist() == [(36 + 21) * 5, (36 + 21) * 6, 0, 0]


def test_structured_jacobian_matches_its_sparsity():
    """The propagation Jacobian's structure: unit rows 3 and 5; row 2 the
    unit diagonal and five values; rows 0, 1, 4 four values (columns 0, 1,
    3, 4).  Derivation of the count of the upper triangle of (J C) J^T:
      * (J C)_im = J_i . C_m: rows 3, 5 are C's rows (free); rows 0, 1, 4
        cost 4 mul + 3 add per entry, row 2 5 mul + 5 add.  Entries needed:
        rows 0, 1, 2 all six; row 4 only m in {0, 1, 3, 4, 5} (the rows j >= 4
        of J reach no other column) -> 98 mul, 81 add;
      * C'_ij = (J C)_i . J_j for i <= j: unit rows j = 3, 5 are free; j in
        {0, 1, 4} costs 4 mul + 3 add, j = 2 5 mul + 5 add, for j + 1 values
        of i -> 47 mul, 39 add;
      * C'_34 = C_3 . J_4 is the same sum of the same products as
        (J C)_43 = J_4 . C_3 (C symmetric, terms in the same order): one
        4 mul + 3 add dot product is shared.
    Total 141 mul, 117 add."""
    J = np.eye(6)
    for r in (0, 1, 4):
        for c in (0, 1, 3, 4):
            J[r, c] = 1.5 + 0.1 * r + 0.01 * c
    for c in (0, 1, 3, 4, 5):
        J[2, c] = 0.3 + 0.05 * c
    assert oracle.census_transport(J, _c21()).tolist() == [81 + 39 - 3, 98 + 47 - 4, 0, 0]


def test_plane_jacobian_matches_its_sparsity():
    """The plane step's Jacobian: unit rows 3 and 5; row 2 zero; row 0 the
    unit x entry and values in columns 2-5, row 1 likewise with its unit y
    entry, row 4 values in columns 2, 3, 5 and its unit phi entry.  Count of
    the upper triangle of (J C) J^T:
      * (J C)_im: rows 0, 1 cost 4 mul + 4 add per entry (the unit term is an
        add), row 4 3 mul + 3 add, rows 2, 3, 5 nothing.  Entries needed:
        row 0 all six, row 1 m in {1..5}, row 4 m in {2..5} -> 56 mul, 56 add;
      * C'_ij for i <= j: j = 2 is zero, j = 3, 5 are entries of J C; j = 0
        (i = 0) and j = 1 (i = 0, 1) cost 4 mul + 4 add, j = 4 (i = 0, 1, 3,
        4) 3 mul + 3 add -> 24 mul, 24 add;
      * C'_34 = C_3 . J_4 is the same sum of the same products as (J C)_43 =
        J_4 . C_3: one 3 mul + 3 add dot product is shared.
    Total 77 mul, 77 add."""
    J = np.eye(6)
    J[2, 2] = 0.0
    for r in (0, 1, 4):
        for c in (2, 3, 5):
            J[r, c] = 1.5 + 0.1 * r + 0.01 * c
    J[0, 4], J[1, 4] = 0.7, 0.8
    assert oracle.census_transport(J, _c21()).tolist() == [77, 77, 0, 0]


def test_a_second_disk_hit_costs_the_hit_work_only():
    """On a disk the hits need no alignment rotation: the residual (2 sub,
    then r-phi and r each 2 mul and 1 add) and the quadratic form (8 mul, 3
    add): 12 mul, 7 add, whatever the hit."""
    from synth import make_batch
    from synth.events import true_hit_lists
    b = make_batch("c5", tracks=60)
    L = b.det.n_layers
    x, y, z, lay = b.event_hits(0)
    lists, n = true_hit_lists(b, 0, b.det.n_surfaces)
    for t in range(len(n)):
        j = next((j for j in range(3, n[t]) if lay[lists[t, j]] >= L), None)
        if j is None:
            continue
        s = int(np.nonzero(b.seed_sim == t)[0][0])
        p, C, _, st = oracle.fit(b.det, b.params[:, s:s + 1], b.cov[:, s:s + 1], lists[t:t + 1], np.array([j]),
                                 x, y, z, lay, align=b.align, ms_after_last=True)
        h = lists[t, j]
        m = np.array([x[h], y[h], z[h]], np.float64)
        c1 = oracle.census_disk_step(b.det, p[0], C[0], int(lay[h]), m, m + np.array([0.05, 0.0, 0.0]))
        c2 = oracle.census_disk_step(b.det, p[0], C[0], int(lay[h]), m, m + np.array([-0.02, 0.03, 0.0]))
        assert c1 is not None and c2 is not None
        assert c1[2].tolist() == [7, 12, 0, 0]
        assert np.array_equal(c1, c2)
        return
    raise AssertionError("no disk step")


def _a_state():
    from synth import make_batch
    b = make_batch("c1", tracks=20)
    x, y, z, lay = b.event_hits(0)
    s = 0
    th = b.track_hits[0][b.seed_sim[s]]
    dec = np.full(b.det.n_layers, -2, np.int32)
    st, _, _, _, p, C = oracle.replay_decisions(b, 0, s, dec)
    h = int(th[3])
    return b, p, C, np.array([x[h], y[h], z[h]], np.float64)


def test_a_second_hit_costs_the_hit_work_only():
    """The frame of a prediction (S, its inverse, the z window) is shared by
    all hits tested against it; a hit adds its alignment rotation (4 mul,
    1 add, 2 sub), its residual (2 sub and 2 mul along the tangent, 1 sub in
    z: 2 mul, 4 add) and the quadratic form (8 mul, 3 add): 14 mul, 10 add,
    whatever the hit."""
    b, p, C, m = _a_state()
    c1 = oracle.census_step(b.det, p, C, 3, m, m + np.array([0.0, 0.0, 0.05]), (1e-3, 1e-3))
    c2 = oracle.census_step(b.det, p, C, 3, m, m + np.array([0.02, -0.01, -0.3]), (1e-3, 1e-3))
    assert c1 is not None and c2 is not None
    assert c1[2].tolist() == [10, 14, 0, 0]
    assert np.array_equal(c1, c2)


def test_stored_counts_match_a_fresh_census():
    from oracle import flop_census
    fresh = flop_census.census()
    stored = flop_census.load()
    for k, v in fresh["flops"].items():
        assert stored["flops"][k] == pytest.approx(v, rel=5e-3), k
    assert stored["window_hits_per_step"] == pytest.approx(fresh["window_hits_per_step"], rel=5e-3)
    fresh_d = flop_census.census_disks()
    for k, v in fresh_d["flops"].items():
        assert stored["disks"]["flops"][k] == pytest.approx(v, rel=5e-3), k
    assert stored["disks"]["window_hits_per_disk_step"] == pytest.approx(fresh_d["window_hits_per_disk_step"],
                                                                          rel=5e-3)
