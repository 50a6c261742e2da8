"""Pins of the FP64 oracle against things other than itself (no GPU).

Each pin is chosen so that a plausible mistake in the oracle (dropped term,
wrong sign or index, transposed operand) fails at least one of them:
closed forms for the gates, a brute-force Kronecker-product unitary, the
state-vector definition, unit norm, slice-sum == uncut, per-slice projector
substitution, the exact shift rule vs finite differences vs the adjoint, and
the paper's worked permutation example.
"""
import itertools
import math

import numpy as np
import pytest
import scipy.linalg

from oracle import gates as G
from oracle import gradients as GR
from oracle import network as NW
from oracle import permute as PM
from oracle import selection as SEL
from oracle import statevector as SV
from qflex_inputs import (c1_problem, grid_lattice, grid_problem,
                          random_bitstrings, random_circuit)
from qflex_inputs.circuits import Circuit, Gate


# ---------------------------------------------------------------- gates
def test_gate_closed_forms():
    assert np.allclose(G.SX @ G.SX, G.X)
    assert np.allclose(G.SY @ G.SY, G.Y)
    assert np.allclose(G.T @ G.T, np.diag([1, 1j]))
    assert np.allclose(G.H @ G.H, np.eye(2))
    for U in (G.H, G.T, G.SX, G.SY, G.CZ):
        assert np.allclose(U.conj().T @ U, np.eye(U.shape[0]))
    assert np.allclose(G.rotation("RX", np.pi), -1j * G.X)
    for kind, P in (("RX", G.X), ("RY", G.Y), ("RZ", G.Z)):
        for th in (0.3, 2.0, 5.9):
            assert np.allclose(G.rotation(kind, th), scipy.linalg.expm(-0.5j * th * P))


def test_cz_schmidt_split_sums_to_cz():
    # (-1)^{ab} = sum_k |k><k|_a (x) Z^k_b, lower-index qubit first
    acc = sum(np.kron(G.cz_half("proj", k), G.cz_half("z", k)) for k in (0, 1))
    assert np.allclose(acc, G.CZ)


# ---------------------------------------------------------------- state vector
def _iswap_ketbra():
    """|00><00| + |11><11| + i|01><10| + i|10><01| (Methods, "Revised set of RQCs")."""
    ket = {b: np.eye(4)[int(b, 2)].reshape(4, 1) for b in ("00", "01", "10", "11")}
    return (ket["00"] @ ket["00"].T + ket["11"] @ ket["11"].T
            + 1j * ket["01"] @ ket["10"].T + 1j * ket["10"] @ ket["01"].T)


def test_iswap_split_sums_to_definition():
    ref = _iswap_ketbra()
    assert np.allclose(G.ISWAP, ref)
    acc = sum(np.kron(G.iswap_half("a", k), G.iswap_half("b", k)) for k in range(4))
    assert np.allclose(acc, ref, atol=1e-15)
    assert np.allclose(ref @ ref.conj().T, np.eye(4))


def _operator_schmidt_rank(U4):
    # U[(a b), (a' b')] -> M[(a a'), (b b')]; its rank is the operator-Schmidt rank
    M = U4.reshape(2, 2, 2, 2).transpose(0, 2, 1, 3).reshape(4, 4)
    return int(np.sum(np.linalg.svd(M, compute_uv=False) > 1e-12))


def test_schmidt_ranks_of_two_qubit_gates():
    # Methods, "Overview of the simulator": 2 for CZ (any diagonal gate), 4 for iSWAP
    assert _operator_schmidt_rank(G.CZ) == 2
    assert _operator_schmidt_rank(_iswap_ketbra()) == 4


def _kron_unitary(circ):
    n = circ.n
    U = np.eye(1 << n, dtype=np.complex128)
    for g in sorted(circ.gates, key=lambda g: g.cycle):
        if g.kind == "CZ":
            d = np.ones(1 << n, dtype=np.complex128)
            for idx in range(1 << n):
                if (idx >> (n - 1 - g.q0)) & 1 and (idx >> (n - 1 - g.q1)) & 1:
                    d[idx] = -1
            M = np.diag(d)
        elif g.kind == "ISWAP":
            # brute force on basis states: |..0_a..1_b..> -> i|..1_a..0_b..> and back
            M = np.zeros((1 << n, 1 << n), dtype=np.complex128)
            ba, bb = n - 1 - g.q0, n - 1 - g.q1
            for idx in range(1 << n):
                xa, xb = (idx >> ba) & 1, (idx >> bb) & 1
                if xa == xb:
                    M[idx, idx] = 1
                else:
                    M[idx ^ (1 << ba) ^ (1 << bb), idx] = 1j
        else:
            ops = [np.eye(2)] * n
            ops[g.q0] = G.single_qubit_matrix(g.kind, circ.angles, g.param)
            M = ops[0]
            for o in ops[1:]:
                M = np.kron(M, o)
        U = M @ U
    return U


@pytest.mark.parametrize("rot,two", [(False, "CZ"), (True, "CZ"), (False, "ISWAP"), (True, "ISWAP")])
def test_statevector_vs_kronecker_unitary(rot, two):
    circ = random_circuit(grid_lattice(2, 3), 10, seed=4, rotations=rot, two_qubit=two)
    U = _kron_unitary(circ)
    psi = SV.final_state(circ).reshape(-1)
    assert np.allclose(psi, U[:, 0], atol=1e-13)


def test_identity_circuit_amplitude():
    circ = random_circuit(grid_lattice(2, 2), 0, seed=0)   # H then H
    psi = SV.final_state(circ).reshape(-1)
    assert abs(psi[0] - 1) < 1e-14 and np.allclose(psi[1:], 0)


# ---------------------------------------------------------------- network
@pytest.mark.parametrize("rows,cols,t,seed", [(2, 2, 8, 0), (2, 3, 12, 1), (3, 3, 16, 2)])
def test_contraction_matches_statevector(rows, cols, t, seed):
    p = grid_problem(rows, cols, t, seed, r0=1, c0=1, cuts=False, tile_rows=1, tile_cols=1)
    bs = random_bitstrings(p.n, 3, seed)
    a = NW.amplitudes(p, bs)
    r = SV.amplitudes(p.circuit, bs, p.open_tile)
    assert np.max(np.abs(a - r)) < 1e-14


@pytest.mark.parametrize("rows,cols,t,seed", [(2, 3, 8, 0), (3, 3, 8, 1), (2, 3, 16, 2)])
def test_iswap_contraction_matches_statevector(rows, cols, t, seed):
    p = grid_problem(rows, cols, t, seed, r0=1, c0=1, cuts=False, tile_rows=1, tile_cols=1,
                     two_qubit="ISWAP")
    bs = random_bitstrings(p.n, 3, seed)
    a = NW.amplitudes(p, bs)
    r = SV.amplitudes(p.circuit, bs, p.open_tile)
    assert np.max(np.abs(a - r)) < 1e-14


def test_iswap_bonds_match_cz_at_twice_the_depth():
    # Methods, "Revised set of RQCs" / "Overview of the simulator": depth
    # 1+t/2+1 with iSWAPs costs what depth 1+t+1 with CZs costs (t/2 a
    # multiple of the 8-cycle layer period, so every edge is covered)
    for t in (16, 32, 48):
        cz = random_circuit(grid_lattice(4, 5), t, 3)
        isw = random_circuit(grid_lattice(4, 5), t // 2, 3, two_qubit="ISWAP")
        assert np.array_equal(NW.bond_exponents(cz), NW.bond_exponents(isw))


def test_iswap_slice_sum_and_per_slice_substitution():
    p = grid_problem(3, 4, 8, 3, r0=2, c0=2, cuts=True, tile_rows=1, tile_cols=2, two_qubit="ISWAP")
    P = NW.n_slices(p.circuit, p.cut_edges)
    assert P == 16                      # two cut edges, one iSWAP (2 bits) each
    bs = random_bitstrings(p.n, 2, 5)
    full = NW.amplitudes(p, bs)
    ref = SV.amplitudes(p.circuit, bs, p.open_tile)
    assert np.max(np.abs(full - ref)) < 1e-15
    for s in (0, 6, 9, 15):
        vals = NW.slice_values(p.circuit, p.cut_edges, s)
        got = NW.slice_amplitudes(p, bs[1], s)
        want = SV.amplitudes(p.circuit, bs[1:], p.open_tile, cut_values=vals)[0]
        assert np.max(np.abs(got - want)) < 1e-15


def test_iswap_planted_mistakes_fail_a_pin(monkeypatch):
    p = grid_problem(3, 4, 8, 3, r0=2, c0=2, cuts=True, tile_rows=1, tile_cols=2, two_qubit="ISWAP")
    bs = random_bitstrings(p.n, 1, 5)
    ref = SV.amplitudes(p.circuit, bs, p.open_tile)
    orig = G.iswap_half
    # (a) a conjugated coefficient (-i/2 for i/2): the full sum moves
    monkeypatch.setattr(G, "iswap_half", lambda role, k: orig(role, k).conj() if role == "b" and k >= 2
                        else orig(role, k))
    assert np.max(np.abs(NW.amplitudes(p, bs) - ref)) > 1e-6
    # (b) the two bits of k swapped in the bond index: the full sum is a
    #     relabelling and still matches, a per-slice value does not
    flip = lambda role, k: orig(role, ((k & 1) << 1) | (k >> 1))
    monkeypatch.setattr(G, "iswap_half", flip)
    assert np.max(np.abs(NW.amplitudes(p, bs) - ref)) < 1e-14
    vals = NW.slice_values(p.circuit, p.cut_edges, 6)
    monkeypatch.setattr(G, "iswap_half", orig)
    want = SV.amplitudes(p.circuit, bs, p.open_tile, cut_values=vals)[0]
    monkeypatch.setattr(G, "iswap_half", flip)
    got = NW.slice_amplitudes(p, bs[0], 6)
    assert np.max(np.abs(got - want)) > 1e-6


def test_c1_full_tile_norm_and_statevector():
    p = c1_problem(0, full_tile=True)
    bs = random_bitstrings(16, 1, 0)
    a = NW.amplitudes(p, bs)[0]
    assert abs(np.sum(np.abs(a) ** 2) - 1.0) < 1e-12
    psi = SV.final_state(p.circuit).reshape(-1)
    assert np.max(np.abs(a - psi)) < 1e-14       # tile = all qubits, qubit 0 most significant


def test_slice_sum_equals_uncut_and_per_slice_substitution():
    p = grid_problem(3, 4, 16, 3, r0=2, c0=2, cuts=True, tile_rows=1, tile_cols=2)
    P = NW.n_slices(p.circuit, p.cut_edges)
    assert P == 16
    bs = random_bitstrings(p.n, 2, 5)
    full = NW.amplitudes(p, bs)
    ref = SV.amplitudes(p.circuit, bs, p.open_tile)
    assert np.max(np.abs(full - ref)) < 1e-15
    for s in (0, 7, 15):
        vals = NW.slice_values(p.circuit, p.cut_edges, s)
        got = NW.slice_amplitudes(p, bs[1], s)
        want = SV.amplitudes(p.circuit, bs[1:], p.open_tile, cut_values=vals)[0]
        assert np.max(np.abs(got - want)) < 1e-15


def test_mixed_radix_first_cut_most_significant():
    p = grid_problem(3, 4, 16, 3, r0=2, c0=2, cuts=True, tile_rows=1, tile_cols=2)
    e0, e1 = p.cut_edges
    assert NW.slice_values(p.circuit, p.cut_edges, 1) == {e0: 0, e1: 1}
    assert NW.slice_values(p.circuit, p.cut_edges, 4) == {e0: 1, e1: 0}


def _circuit_2x2(body):
    """2x2 grid (edges (0,1), (0,2), (1,3), (2,3)) with the given gates."""
    lat = grid_lattice(2, 2)
    return Circuit(lat, 4, list(body), np.zeros(0)), lat.edge_index


def _assert_zero_rule_against_statevector(circ, cuts):
    """Every path the projector rule rules out is the zero vector under the
    state-vector substitution of its cut values; every other path is not;
    the kept paths sum to the uncut state."""
    nz = set(NW.nonzero_slices(circ, cuts))
    total = np.zeros((2,) * circ.n, dtype=np.complex128)
    for s in range(NW.n_slices(circ, cuts)):
        psi = SV.final_state(circ, cut_values=NW.slice_values(circ, cuts, s))
        if s in nz:
            assert np.linalg.norm(psi) > 1e-6, s
            total += psi
        else:
            assert np.max(np.abs(psi)) == 0.0, s
    assert np.max(np.abs(total - SV.final_state(circ))) < 1e-14
    return nz


def test_structurally_zero_paths_closed_forms():
    """Closed forms of the projector rule (P_j P_k = delta_jk P_k through
    diagonal gates; P_k |0> = delta_k0 |0>) on hand-made 2x2 circuits."""
    H = lambda c, qs=range(4): [Gate(c, "H", q) for q in qs]
    # qubit 0 is the projector side of (0,1) and (0,2); only T between them
    circ, ei = _circuit_2x2(H(0) + [Gate(1, "CZ", 0, 1), Gate(2, "T", 0), Gate(3, "CZ", 0, 2)] + H(4))
    cuts = [ei[(0, 1)], ei[(0, 2)]]
    assert _assert_zero_rule_against_statevector(circ, cuts) == {0, 3}
    # a non-diagonal gate between them: no constraint
    circ, ei = _circuit_2x2(H(0) + [Gate(1, "CZ", 0, 1), Gate(2, "SX", 0), Gate(3, "CZ", 0, 2)] + H(4))
    assert _assert_zero_rule_against_statevector(circ, cuts) == {0, 1, 2, 3}
    # qubit 3 is the Z side of (1,3) and (2,3): Z halves never vanish
    circ, ei = _circuit_2x2(H(0) + [Gate(1, "CZ", 1, 3), Gate(2, "RZ", 3, param=0), Gate(3, "CZ", 2, 3)] + H(4))
    circ = circ.with_angles(np.array([0.7]))
    assert _assert_zero_rule_against_statevector(circ, [ei[(1, 3)], ei[(2, 3)]]) == {0, 1, 2, 3}
    # a projector before qubit 0's first non-diagonal gate acts on |0>
    circ, ei = _circuit_2x2(H(0, (1, 2, 3)) + [Gate(1, "CZ", 0, 1), Gate(2, "H", 0)] + H(3))
    assert _assert_zero_rule_against_statevector(circ, [ei[(0, 1)]]) == {0}
    # two CZs on one edge with RZ between: its two bits agree (values 00, 11)
    circ, ei = _circuit_2x2(H(0) + [Gate(1, "CZ", 0, 1), Gate(2, "RZ", 0, param=0), Gate(3, "CZ", 0, 1)] + H(4))
    circ = circ.with_angles(np.array([1.3]))
    assert _assert_zero_rule_against_statevector(circ, [ei[(0, 1)]]) == {0, 3}


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_structurally_zero_paths_random_circuits(seed):
    """3x3, 1+16+1, cuts on the two bonds whose projector side is the centre
    qubit and one more: the rule removes some paths, and the state vector
    confirms each removed path vanishes and the rest sum to the state."""
    circ = random_circuit(grid_lattice(3, 3), 16, seed)
    ei = circ.lattice.edge_index
    cuts = [ei[(4, 5)], ei[(4, 7)], ei[(1, 2)]]
    nz = _assert_zero_rule_against_statevector(circ, cuts)
    assert len(nz) < NW.n_slices(circ, cuts)


def test_structurally_zero_planted_mistakes_fail(monkeypatch):
    """A rule that also treats X^1/2 and Y^1/2 as diagonal, or that forgets
    the input |0>, disagrees with the state vector."""
    circ = random_circuit(grid_lattice(3, 3), 16, 0)
    ei = circ.lattice.edge_index
    cuts = [ei[(4, 5)], ei[(4, 7)], ei[(1, 2)]]
    monkeypatch.setattr(NW, "_DIAGONAL_1Q", ("T", "RZ", "SX", "SY"))
    with pytest.raises(AssertionError):
        _assert_zero_rule_against_statevector(circ, cuts)
    monkeypatch.setattr(NW, "_DIAGONAL_1Q", ("T", "RZ"))
    H = lambda c, qs=range(4): [Gate(c, "H", q) for q in qs]
    circ, ei = _circuit_2x2(H(0, (1, 2, 3)) + [Gate(1, "CZ", 0, 1), Gate(2, "H", 0)] + H(3))
    orig = NW.projector_runs
    monkeypatch.setattr(NW, "projector_runs", lambda c, cu: (orig(c, cu)[0], [False] * len(orig(c, cu)[1])))
    with pytest.raises(AssertionError):
        _assert_zero_rule_against_statevector(circ, [ei[(0, 1)]])


def test_planted_mistakes_fail_a_pin(monkeypatch):
    """Plant plausible mistakes in the oracle's CZ split; a pin catches each."""
    p = grid_problem(2, 3, 12, 1, r0=1, c0=1, cuts=True, tile_rows=1, tile_cols=1)
    bs = random_bitstrings(p.n, 1, 2)
    ref = SV.amplitudes(p.circuit, bs, p.open_tile)
    orig = G.cz_half
    # (a) a dropped sign: Z^k replaced by the identity -> the amplitude changes
    monkeypatch.setattr(G, "cz_half", lambda role, k: orig("proj", k) if role == "proj" else np.eye(2))
    assert np.max(np.abs(NW.amplitudes(p, bs) - ref)) > 1e-6
    # (b) swapped split orientation: the full sum still matches, but a per-slice
    #     value no longer equals the substituted state vector (which keeps the
    #     stated orientation)
    monkeypatch.setattr(G, "cz_half", lambda role, k: orig("z" if role == "proj" else "proj", k))
    assert np.max(np.abs(NW.amplitudes(p, bs) - ref)) < 1e-14
    vals = NW.slice_values(p.circuit, p.cut_edges, 1)
    monkeypatch.setattr(G, "cz_half", orig)
    want = SV.amplitudes(p.circuit, bs, p.open_tile, cut_values=vals)[0]
    monkeypatch.setattr(G, "cz_half", lambda role, k: orig("z" if role == "proj" else "proj", k))
    got = NW.slice_amplitudes(p, bs[0], 1)
    assert np.max(np.abs(got - want)) > 1e-6


# ---------------------------------------------------------------- gradients
def test_shift_rule_fd_and_adjoint_agree():
    circ = random_circuit(grid_lattice(2, 3), 12, seed=7, rotations=True)
    bs = random_bitstrings(circ.n, 1, 3)
    tile = [4, 5]

    def amp(th):
        return SV.amplitudes(circ, bs, tile, angles=th)[0]

    params = list(range(circ.n_params))
    sr = GR.shift_rule(amp, circ.angles, params)
    fd = GR.finite_difference(amp, circ.angles, params)
    assert np.max(np.abs(sr - fd)) < 1e-8
    g = (np.random.default_rng(0).normal(size=4) + 1j * np.random.default_rng(1).normal(size=4))
    adj = GR.statevector_adjoint(circ, bs, tile, g)
    assert np.max(np.abs(adj - GR.loss_gradient(sr, g))) < 1e-12


def test_iswap_rotation_gradients_agree():
    circ = random_circuit(grid_lattice(2, 3), 8, seed=11, rotations=True, two_qubit="ISWAP")
    bs = random_bitstrings(circ.n, 1, 3)
    tile = [3, 4]

    def amp(th):
        return SV.amplitudes(circ, bs, tile, angles=th)[0]

    params = list(range(circ.n_params))
    sr = GR.shift_rule(amp, circ.angles, params)
    fd = GR.finite_difference(amp, circ.angles, params)
    assert np.max(np.abs(sr - fd)) < 1e-8
    g = (np.random.default_rng(2).normal(size=4) + 1j * np.random.default_rng(3).normal(size=4))
    adj = GR.statevector_adjoint(circ, bs, tile, g)
    assert np.max(np.abs(adj - GR.loss_gradient(sr, g))) < 1e-12


def test_network_shift_rule_matches_statevector():
    p = grid_problem(2, 3, 12, 9, r0=1, c0=1, cuts=True, tile_rows=1, tile_cols=1, rotations=True)
    bs = random_bitstrings(p.n, 1, 4)
    params = [0, 5, p.circuit.n_params - 1]
    tn = GR.shift_rule(lambda th: NW.amplitudes(p, bs, angles=th)[0], p.circuit.angles, params)
    sv = GR.shift_rule(lambda th: SV.amplitudes(p.circuit, bs, p.open_tile, angles=th)[0],
                       p.circuit.angles, params)
    assert np.max(np.abs(tn - sv)) < 1e-14


# ---------------------------------------------------------------- permutation
def _brute_permute(x, perm):
    out = np.empty([x.shape[p] for p in perm], dtype=x.dtype)
    for j in itertools.product(*[range(d) for d in out.shape]):
        i = [0] * x.ndim
        for a, p in enumerate(perm):
            i[p] = j[a]
        out[j] = x[tuple(i)]
    return out


def test_permute_definition_brute_force():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(2, 3, 4, 2)) + 1j * rng.normal(size=(2, 3, 4, 2))
    for perm in ([3, 1, 0, 2], [0, 1, 2, 3], [2, 3, 1, 0]):
        assert np.array_equal(PM.permute(x, perm), _brute_permute(x, perm))


def test_paper_worked_permutation_example():
    """abcdefg -> cfeadgb through L2 (abc|de|fg -> cae|bd|fg), R4 (-> cae|fd|gb),
    L2 (-> cfe|ad|gb), as worked in Methods, "Cache-efficient index permutations"."""
    rng = np.random.default_rng(1)
    order = list("abcdefg")
    x = rng.normal(size=(2,) * 7) + 1j * rng.normal(size=(2,) * 7)
    s1, s2, s3 = list("caebdfg"), list("caefdgb"), list("cfeadgb")
    y = PM.apply_move(x, order, s1, "L", 2)
    y = PM.apply_move(y, s1, s2, "R", 4)
    y = PM.apply_move(y, s2, s3, "L", 2)
    direct = PM.permute(x, [order.index(c) for c in s3])
    assert np.array_equal(y, direct)
    with pytest.raises(ValueError):             # an L move may not touch the right group
        PM.apply_move(x, order, list("abcdegf"), "L", 2)
    moves = PM.lr_decompose(order, s3, 2, 4)
    assert [m[:2] for m in moves] == [("L", 2), ("R", 4), ("L", 2)]
    assert np.array_equal(PM.permute_lr(x, order, s3, 2, 4), direct)


def test_lr_decomposition_random_binary_perms():
    rng = np.random.default_rng(2)
    n = 12
    labels = [chr(ord("a") + i) for i in range(n)]
    x = rng.normal(size=(2,) * n).astype(np.complex128)
    for _ in range(10):
        tgt = list(rng.permutation(labels))
        want = PM.permute(x, [labels.index(c) for c in tgt])
        assert np.array_equal(PM.permute_lr(x, labels, tgt, 3, 6), want)


# ---------------------------------------------------------------- selection
def test_splitmix64_published_vector():
    r = SEL.SplitMix64(0)
    assert [r.next() for _ in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                           0x06C45D188009454F]


def test_fraction_selection():
    assert SEL.n_selected(0.01, 65536) == 655
    assert SEL.n_selected(0.5 / 1024, 1024) == 1          # 0.5 rounds half up
    assert SEL.n_selected(1e-9, 1024) == 1
    assert SEL.n_selected(2.0, 16) == 16
    s = SEL.select_slices(1024, 0.1, 42)
    assert len(s) == 102 and s == sorted(set(s)) and s == SEL.select_slices(1024, 0.1, 42)
    assert s != SEL.select_slices(1024, 0.1, 43)
    # every slice is equally likely: counts over seeds stay near their mean
    cnt = np.zeros(64)
    for seed in range(2000):
        cnt[SEL.select_slices(64, 0.25, seed)] += 1
    assert cnt.min() > 0.8 * 500 and cnt.max() < 1.2 * 500


def test_all_slices_give_unit_norm_and_fraction_norm_is_reported():
    p = grid_problem(3, 4, 16, 3, r0=2, c0=2, cuts=True, tile_rows=3, tile_cols=4)
    bs = random_bitstrings(p.n, 1, 0)
    full = NW.amplitudes(p, bs)[0]                   # tile = all 12 qubits
    assert abs(np.sum(np.abs(full) ** 2) - 1) < 1e-12
    part = NW.amplitudes(p, bs, slices=SEL.select_slices(16, 0.25, 1))[0]
    nrm = float(np.sum(np.abs(part) ** 2))
    assert 0.0 < nrm < 1.0                           # norm ~ f; value is reported, not gated
    f = SEL.overlap_fidelity(full, part)
    assert 0.0 < f <= 1.0 + 1e-12
    assert abs(SEL.overlap_fidelity(full, full) - 1.0) < 1e-12   # all paths: fidelity 1


def test_overlap_fidelity_closed_forms():
    """Eq. fidelity_1 / fidelity_2 (Methods, "Summing a fraction of the
    paths"): F = |<psi|psi~>|^2 / <psi~|psi~>.  Hand cases: the uniform
    2-qubit state and its partial sum over two basis states give F = 1/2
    (<psi|psi~> = 1/2, <psi~|psi~> = 1/2); a state split into P orthogonal
    parts of equal weight, summed over k of them, gives F = k / P exactly;
    a global phase on either side leaves F unchanged."""
    psi = np.full(4, 0.5, dtype=np.complex128)
    part = np.array([0.5, 0.5, 0.0, 0.0], dtype=np.complex128)
    assert abs(SEL.overlap_fidelity(psi, part) - 0.5) < 1e-15
    assert abs(SEL.overlap_fidelity(psi * 1j, part * np.exp(0.3j)) - 0.5) < 1e-15
    rng = np.random.default_rng(4)
    P, n = 8, 64
    parts = np.zeros((P, n), dtype=np.complex128)
    for s in range(P):                            # disjoint supports: orthogonal parts
        v = rng.normal(size=n // P) + 1j * rng.normal(size=n // P)
        parts[s, s * (n // P):(s + 1) * (n // P)] = v / np.linalg.norm(v) / np.sqrt(P)
    full = parts.sum(axis=0)
    for k in (1, 3, 8):
        assert abs(SEL.overlap_fidelity(full, parts[:k].sum(axis=0)) - k / P) < 1e-12


def test_frugal_sampling_acceptance_closed_form():
    """Methods, "Fast sampling technique": with Porter-Thomas amplitudes the
    probability that a batch of N_C yields a sample is 1 - (1 - 1/M)^N_C
    (95.76% for M = 10, N_C = 30); at most one sample per batch, and the
    accepted entries are distributed as min(1, pN/M)-weighted draws."""
    n = 20
    rng = np.random.default_rng(11)
    nb, nc = 3000, 30
    amps = (rng.standard_normal((nb, nc)) + 1j * rng.standard_normal((nb, nc))) * np.sqrt(0.5 * 2.0 ** -n)
    acc = SEL.frugal_sample(amps, n, 10.0, seed=5)
    rate = float(np.mean(acc >= 0))
    assert abs(rate - (1 - (1 - 0.1) ** 30)) < 0.012
    assert np.all((acc >= -1) & (acc < nc))
    # a batch of zeros never accepts; a batch with one entry p N >= M always does
    z = np.zeros((1, 8), dtype=np.complex128)
    assert SEL.frugal_sample(z, n, 10.0, 1)[0] == -1
    z[0, 5] = np.sqrt(20.0 * 2.0 ** -n)
    assert SEL.frugal_sample(z, n, 10.0, 1)[0] == 5
    # accepted samples favour large |amp|^2 (mean p N of accepted > 1)
    p = np.abs(amps) ** 2 * 2.0 ** n
    sel = acc[acc >= 0]
    assert np.mean(p[np.arange(nb)[acc >= 0], sel]) > 1.5


# ---------------------------------------------------------------- fidelity-f samples
def test_fidelity_samples_special_cases_and_rates():
    """Methods, "Fraction of perfect fidelity amplitudes": f = 1 takes only
    exact samples (accepted batches, in batch order, tile bits from the
    accepted index); f = 0 only uniform bitstrings; otherwise the exact
    fraction is Binomial(n, f) and uniform bits are fair and independent."""
    rng = np.random.default_rng(3)
    n, nb, tile = 70, 4000, [60, 61, 62, 63, 64, 65]
    bits = rng.integers(0, 2, size=(nb, n), dtype=np.uint8)
    acc = rng.integers(-1, 64, size=nb).astype(np.int32)
    pool = np.flatnonzero(acc >= 0)
    s1, src1, k1 = SEL.fidelity_samples(bits, acc, tile, 1.0, 9, 500)
    assert k1 == 500 and np.array_equal(src1, pool[:500])
    for i in (0, 77, 499):
        b = pool[i]
        want = bits[b].copy()
        for t, q in enumerate(tile):
            want[q] = (acc[b] >> (5 - t)) & 1
        assert np.array_equal(s1[i], want)
    s0, src0, k0 = SEL.fidelity_samples(bits, acc, tile, 0.0, 9, 20000)
    assert k0 == 0 and np.all(src0 == -1)
    sd = 0.5 / np.sqrt(20000)
    assert np.max(np.abs(s0.mean(axis=0) - 0.5)) < 5 * sd
    # independence across the 64-bit word boundary (qubits 63 and 64) and within a word
    for a, b in ((63, 64), (0, 1), (10, 69)):
        assert abs(np.mean(s0[:, a] ^ s0[:, b]) - 0.5) < 5 * sd
    f = 0.37
    _, src, k = SEL.fidelity_samples(bits, acc, tile, f, 4, 3000)
    sd = np.sqrt(f * (1 - f) / 3000)
    assert abs(k / 3000 - f) < 5 * sd and np.sum(src >= 0) == k
    # too few accepted batches: the surplus exact samples are marked -2
    _, src, k = SEL.fidelity_samples(bits[:10], acc[:10], tile, 1.0, 4, 20)
    assert k == 20 and np.sum(src == -2) == 20 - np.sum(acc[:10] >= 0)


@pytest.mark.parametrize("f", [0.25, 0.6])
def test_fidelity_samples_linear_xeb_equals_f(f):
    """The mixture's linear XEB, N <p(x)> - 1, is f times that of exact
    samples (uniform samples contribute 0), and exact samples of a
    Porter-Thomas circuit give N sum p^2 - 1 ~ 1.  Exact samples here come
    from frugal rejection over 64-entry open-tile batches of state-vector
    amplitudes of a 12-qubit RQC."""
    p_ = grid_problem(3, 4, 24, 5, r0=1, c0=2, cuts=False, tile_rows=2, tile_cols=3)
    n = p_.n
    psi = SV.final_state(p_.circuit)
    prob = np.abs(psi.reshape(-1)) ** 2
    nb = 12000
    bits = random_bitstrings(n, nb, 21)
    amps = np.stack([SV.tile_amplitudes_from_state(psi, b, p_.open_tile) for b in bits])
    acc = SEL.frugal_sample(amps, n, 10.0, seed=8)
    ns = 16000
    samples, src, k = SEL.fidelity_samples(bits, acc, p_.open_tile, f, 31, ns)
    assert np.all(src >= -1)
    idx = samples.astype(np.int64) @ (1 << np.arange(n - 1, -1, -1))
    xeb = SEL.linear_xeb(prob[idx], n)
    exact_xeb = SEL.linear_xeb(prob[idx[src >= 0]], n)
    ideal = (2.0 ** n) * np.sum(prob ** 2) - 1.0
    assert abs(exact_xeb - ideal) < 0.1 * ideal
    # N p(x) has variance ~2 under Porter-Thomas: 5 sigma over ns samples
    assert abs(xeb - f * exact_xeb) < 5 * np.sqrt(2.0 / ns) + 5 * np.sqrt(f * (1 - f) / ns) * exact_xeb
    assert abs(xeb - f * ideal) < 0.1 * ideal
