"""Host-side checks of libvqe that need no GPU: the library builds and loads,
exports every function include/vqe.h declares, its Jordan-Wigner mapping agrees
with the oracle's independent one, and it rejects bad arguments."""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from paper_2311_01242_gb300 import _native, api


@pytest.fixture(scope="module")
def lib():
    _native.build()
    return _native.load()


def test_exports_every_declared_symbol(lib):
    names = _native.declared_symbols()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(_native.PROTOTYPES), set(names) ^ set(_native.PROTOTYPES)


def test_version_and_error_message(lib):
    assert lib.vqe_version() >= 100
    assert isinstance(lib.vqe_last_error(), bytes)


@pytest.mark.parametrize("seed,n_s,n_elec", [(0, 2, 2), (1, 3, 2), (2, 4, 4), (3, 6, 6)])
def test_jordan_wigner_matches_oracle(lib, seed, n_s, n_elec):
    prob = synth.random_problem(np.random.default_rng(seed), n_s, n_elec, 3)
    x1, z1, c1 = api.jordan_wigner(prob.n_spatial, prob.h, prob.eri)
    x2, z2, c2 = oracle.jordan_wigner(prob)
    assert np.array_equal(x1, x2) and np.array_equal(z1, z2)
    assert np.abs(c1 - c2).max() < 1e-12


def test_jordan_wigner_config1_and_drop(lib):
    prob = synth.config1(1).problems[0]
    x1, z1, c1 = api.jordan_wigner(prob.n_spatial, prob.h, prob.eri)
    x2, z2, c2 = oracle.jordan_wigner(prob)
    assert len(x1) == len(x2) == 1819 and len(set(x1.tolist())) == 286
    assert np.abs(c1 - c2).max() < 1e-12
    xd, zd, cd = api.jordan_wigner(prob.n_spatial, prob.h, prob.eri, 0.0, 1e-2)
    keep = np.abs(c2) >= 1e-2
    assert np.array_equal(xd, x2[keep]) and np.array_equal(zd, z2[keep])


def test_jordan_wigner_constant_and_capacity(lib):
    prob = synth.config0().problems[0]
    x, z, c = api.jordan_wigner(2, prob.h, prob.eri, c0=1.25)
    x0, z0, c0 = api.jordan_wigner(2, prob.h, prob.eri, c0=0.0)
    ident = (x == 0) & (z == 0)
    ident0 = (x0 == 0) & (z0 == 0)
    assert abs(c[ident][0] - c0[ident0][0] - 1.25) < 1e-14
    n = ctypes.c_int64(0)
    h = np.ascontiguousarray(prob.h)
    e = np.ascontiguousarray(prob.eri)
    rc = lib.vqe_jordan_wigner(2, api._ptr(h), api._ptr(e), 0.0, 0.0, 3, None, None, None, ctypes.byref(n))
    assert rc == 1 and n.value == len(x0)


def test_jordan_wigner_rejects_bad_input(lib):
    n = ctypes.c_int64(0)
    h = np.zeros((2, 2))
    e = np.zeros((2, 2, 2, 2))
    assert lib.vqe_jordan_wigner(0, api._ptr(h), api._ptr(e), 0.0, 0.0, 0, None, None, None,
                                 ctypes.byref(n)) == 1
    hn = h.copy()
    hn[0, 1] = np.nan
    assert lib.vqe_jordan_wigner(2, api._ptr(hn), api._ptr(e), 0.0, 0.0, 0, None, None, None,
                                 ctypes.byref(n)) == 1
    assert b"non-finite" in lib.vqe_last_error()
    # an antisymmetric one-body matrix maps to imaginary coefficients
    ha = np.array([[0.0, 1.0], [-1.0, 0.0]])
    assert lib.vqe_jordan_wigner(2, api._ptr(ha), api._ptr(e), 0.0, 0.0, 0, None, None, None,
                                 ctypes.byref(n)) == 5


def test_create_rejects_invalid_arguments_before_device_work(lib):
    h = ctypes.c_void_p()
    xs = np.array([1 << 5], dtype=np.uint64)
    zs = np.array([0], dtype=np.uint64)
    cs = np.array([1.0])
    assert lib.vqe_create_hamiltonian(4, 1, api._ptr(xs), api._ptr(zs), api._ptr(cs), 0.0,
                                      ctypes.byref(h)) == 1
    assert b"mask bit" in lib.vqe_last_error()
    assert lib.vqe_create_hamiltonian(33, 1, api._ptr(xs), api._ptr(zs), api._ptr(cs), 0.0,
                                      ctypes.byref(h)) == 1
    a = ctypes.c_void_p()
    exc = np.array([[0, 1, 1, 2]], dtype=np.int32)
    assert lib.vqe_create_ansatz(4, 3, 1, api._ptr(exc), ctypes.byref(a)) == 1
    assert b"repeats" in lib.vqe_last_error()
    exc = np.array([[0, 7, -1, -1]], dtype=np.int32)
    assert lib.vqe_create_ansatz(4, 3, 1, api._ptr(exc), ctypes.byref(a)) == 1
    assert lib.vqe_create_ansatz(4, 1 << 6, 0, None, ctypes.byref(a)) == 1


def test_mlp_param_count_matches_oracle_layout(lib):
    from oracle import mlp as omlp
    for dims in [(9, 256, 360), (3, 16, 5), (17, 32, 16)]:
        assert lib.vqe_mlp_param_count(*dims) == omlp.layout(*dims)[1]
    assert lib.vqe_mlp_param_count(9, 20, 5) == 0  # hidden width must be a multiple of 16
    assert lib.vqe_mlp_workspace_bytes(128, 9, 256, 360) > 0


@pytest.mark.parametrize("seed,n_s,n_pairs", [(90, 2, 1), (91, 4, 2), (92, 6, 3), (93, 7, 2)])
def test_hcb_hamiltonian_matches_oracle_block(lib, seed, n_s, n_pairs):
    """vqe_hcb_hamiltonian's Pauli sum, restricted to n_pairs occupied qubits,
    equals the oracle's seniority-zero block of Eq. 2 (built from the ladder
    operators), and it conserves the pair number."""
    prob = synth.random_problem(np.random.default_rng(seed), n_s, 2 * n_pairs, 3)
    prob.c0 = 0.25
    xs, zs, cs = api.hcb_hamiltonian(n_s, prob.h, prob.eri, prob.c0)
    dense = oracle.pauli_sum_dense(xs, zs, cs, n_s)
    block, bos = oracle.hcb_hamiltonian_matrix(prob, n_pairs)
    idx = bos.astype(np.int64)
    assert np.abs(dense[np.ix_(idx, idx)] - block.toarray()).max() < 1e-12
    ks = np.arange(1 << n_s)
    pc = np.array([bin(k).count("1") for k in ks])
    assert np.abs(dense[pc[:, None] != pc[None, :]]).max() == 0.0


def test_hcb_ansatz_rejects_bad_pairs(lib):
    a = ctypes.c_void_p()
    pairs = np.array([[1, 1]], dtype=np.int32)
    assert lib.vqe_create_ansatz_hcb(4, 3, 1, api._ptr(pairs), ctypes.byref(a)) == 1
    pairs = np.array([[0, 9]], dtype=np.int32)
    assert lib.vqe_create_ansatz_hcb(4, 3, 1, api._ptr(pairs), ctypes.byref(a)) == 1
    assert lib.vqe_create_ansatz_hcb(33, 3, 0, None, ctypes.byref(a)) == 1


@pytest.mark.parametrize("seed,n_s,n_elec,frozen,active", [(120, 5, 6, [0], [1, 2, 3, 4]),
                                                           (121, 6, 8, [0, 1], [2, 3, 4, 5]),
                                                           (122, 6, 6, [0, 2], [1, 3, 5]),
                                                           (123, 4, 4, [], [3, 1, 0, 2])])
def test_fold_frozen_matches_oracle(lib, seed, n_s, n_elec, frozen, active):
    prob = synth.random_problem(np.random.default_rng(seed), n_s, n_elec, 3)
    prob.c0 = -0.5
    h2, e2, c2 = api.fold_frozen(prob.h, prob.eri, prob.c0, frozen, active)
    red = oracle.fold_frozen(prob, frozen, active)
    assert np.abs(h2 - red.h).max() < 1e-13
    assert np.array_equal(e2, red.eri)
    assert abs(c2 - red.c0) < 1e-12


def test_fold_frozen_rejects_overlap_and_range(lib):
    h = np.zeros((3, 3))
    e = np.zeros((3, 3, 3, 3))
    with pytest.raises(api.VQEError):
        api.fold_frozen(h, e, 0.0, [0], [0, 1])
    with pytest.raises(api.VQEError):
        api.fold_frozen(h, e, 0.0, [5], [0, 1])


def test_frozen_core_then_boson_mapping_matches_oracle(lib):
    """The paper's CH3F pipeline in small: freeze the core (Eq. 3), then map the
    active space to pUCCD's boson form. Library host mappings against the oracle's
    fold and its seniority-zero block of the folded problem."""
    prob = synth.random_problem(np.random.default_rng(124), 6, 8, 3)
    frozen, active = [0], [1, 2, 3, 4, 5]
    h2, e2, c2 = api.fold_frozen(prob.h, prob.eri, prob.c0, frozen, active)
    xs, zs, cs = api.hcb_hamiltonian(len(active), h2, e2, c2)
    red = oracle.fold_frozen(prob, frozen, active)
    block, bos = oracle.hcb_hamiltonian_matrix(red, 3)
    dense = oracle.pauli_sum_dense(xs, zs, cs, len(active))
    idx = bos.astype(np.int64)
    assert np.abs(dense[np.ix_(idx, idx)] - block.toarray()).max() < 1e-12
