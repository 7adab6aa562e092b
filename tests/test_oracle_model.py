"""Pins of oracle.model (exact diagonalisation) against facts independent of it."""
import itertools
import math
import os

import numpy as np
import pytest

from oracle import model

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

CASES = [(2, 3, 1 / 3, 0.7, 2), (2, 4, 0.25, 1.0, 3), (3, 3, 1 / 3, 1.3, 3), (2, 5, 0.2, 1.0, 4)]


@pytest.mark.parametrize("lx,ly,flux,v,n", CASES)
def test_mixed_and_real_spectra_equal(lx, ly, flux, v, n):
    """The Fourier transform around the ring is a unitary change of single-particle basis,
    so H_real (Eq. H_real) and the k-space H (Eqs. H_kin, H_k_int) share their spectrum."""
    er = np.linalg.eigvalsh(model.real_space_hamiltonian(lx, ly, flux, 1.0, v, n))
    em = np.linalg.eigvalsh(model.mixed_space_hamiltonian(lx, ly, flux, 1.0, v, n))
    assert np.max(np.abs(er - em)) < 1e-12


def test_config1_spectra_equal():
    """4 x 4 cylinder, flux 1/4, V = 1, N = 4 (1820 states)."""
    er = np.linalg.eigvalsh(model.real_space_hamiltonian(4, 4, 0.25, 1.0, 1.0, 4))
    em = np.linalg.eigvalsh(model.mixed_space_hamiltonian(4, 4, 0.25, 1.0, 1.0, 4))
    assert len(er) == math.comb(16, 4)
    assert np.max(np.abs(er - em)) < 1e-11


@pytest.mark.parametrize("lx,ly,flux,v,n", CASES)
def test_mixed_hamiltonian_real_and_hermitian(lx, ly, flux, v, n):
    """Sec. IV.D: the mixed-basis many-body matrix elements are real."""
    h = model.mixed_space_hamiltonian(lx, ly, flux, 1.0, v, n)
    assert np.max(np.abs(h.imag)) < 1e-14
    assert np.max(np.abs(h - h.conj().T)) < 1e-14
    hr = model.real_space_hamiltonian(lx, ly, flux, 1.0, v, n)
    assert np.max(np.abs(hr - hr.conj().T)) < 1e-14


@pytest.mark.parametrize("lx,ly,flux", [(2, 3, 1 / 3), (4, 4, 0.25), (3, 6, 1 / 6), (5, 2, 0.5)])
def test_single_particle_closed_form(lx, ly, flux):
    """Levels of the Lx x Ly one-body hopping matrix = union over m of the tridiagonal
    h_m with diagonal -2t cos(k_m + x phi) (Eq. H_kin)."""
    a = model.single_particle_levels_real(lx, ly, flux, 1.0)
    b = model.single_particle_levels_momentum(lx, ly, flux, 1.0)
    assert np.max(np.abs(a - b)) < 1e-12


@pytest.mark.parametrize("lx,ly,flux,n", [(2, 4, 0.25, 3), (4, 4, 0.25, 4), (3, 3, 1 / 3, 4)])
def test_free_fermion_ground_energy(lx, ly, flux, n):
    """V = 0: the many-body ground energy is the sum of the N lowest levels."""
    for h in (model.real_space_hamiltonian(lx, ly, flux, 1.0, 0.0, n),
              model.mixed_space_hamiltonian(lx, ly, flux, 1.0, 0.0, n)):
        assert abs(model.ground_energy(h) - model.free_fermion_ground_energy(lx, ly, flux, 1.0, n)) < 1e-11


@pytest.mark.parametrize("lx,ly,flux", [(3, 4, 0.25), (2, 5, 0.2)])
def test_one_particle_is_lowest_level(lx, ly, flux):
    levels = model.single_particle_levels_momentum(lx, ly, flux, 1.0)
    for h in (model.real_space_hamiltonian(lx, ly, flux, 1.0, 2.0, 1),
              model.mixed_space_hamiltonian(lx, ly, flux, 1.0, 2.0, 1)):
        assert abs(model.ground_energy(h) - levels[0]) < 1e-12


@pytest.mark.parametrize("lx,ly,n", [(2, 4, 3), (3, 3, 4), (2, 5, 5)])
def test_atomic_limit_classical_minimum(lx, ly, n):
    """t = 0: H is the classical repulsion V * (number of occupied nearest-neighbour
    bonds); its minimum over all placements, found by brute force, is the ground energy of
    both the real-space and the mixed-space Hamiltonian."""
    bonds = []
    for x in range(lx):
        for y in range(ly):
            if x + 1 < lx:
                bonds.append((x * ly + y, (x + 1) * ly + y))
            bonds.append((x * ly + y, x * ly + (y + 1) % ly))
    best = min(sum(1 for a, b in bonds if a in occ and b in occ)
               for occ in map(set, itertools.combinations(range(lx * ly), n)))
    v = 1.7
    for h in (model.real_space_hamiltonian(lx, ly, 0.3, 0.0, v, n),
              model.mixed_space_hamiltonian(lx, ly, 0.3, 0.0, v, n)):
        assert abs(model.ground_energy(h) - v * best) < 1e-11


def test_fig10_worked_element():
    """Sec. IV.D, Fig. 10(a): the term c+_0 c_2 c_4 c+_6 on an L = 8 ring has coefficient
    (V/L) 2 (cos 2a - cos 4a) = 0.25 (V = 1). The printed type A/B formula
    2[cos l - cos(m + l)] would give 0 here; the figure's value is the one matched."""
    with open(os.path.join(GOLDEN, "fig10_element.txt")) as f:
        line = [ln for ln in f if ln.strip() and not ln.startswith("#")][0].split()
    ly, v = int(line[0]), float(line[1])
    cre = [int(c) for c in line[2].split(",")]
    ann = [int(c) for c in line[3].split(",")]
    expect = float(line[4])
    full = model.fock_basis(ly, 2)
    h = model.mixed_space_hamiltonian(1, ly, 0.0, 1.0, v, 2, basis=full)
    i = np.searchsorted(full, np.uint64(sum(1 << o for o in ann)))
    f = np.searchsorted(full, np.uint64(sum(1 << o for o in cre)))
    assert abs(abs(h[f, i]) - expect) < 1e-14
    a = 2 * math.pi / ly
    assert abs(expect - v / ly * 2 * (math.cos(2 * a) - math.cos(4 * a))) < 1e-15


def test_ground_state_momentum_sector():
    """The mixed-basis Hamiltonian conserves K = sum m n_m mod Ly (Sec. II): it has no
    matrix element between Fock states of different K."""
    lx, ly, n = 3, 4, 3
    basis = model.fock_basis(lx * ly, n)
    h = model.mixed_space_hamiltonian(lx, ly, 0.25, 1.0, 1.0, n, basis=basis)
    ks = np.array([model.total_momentum(lx, ly, int(s)) for s in basis])
    rows, cols = np.nonzero(np.abs(h) > 1e-14)
    assert np.all(ks[rows] == ks[cols])
