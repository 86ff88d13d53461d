"""Independent reference constructions for pinning the oracle.

Spin-1/2 Hamiltonians are built as sums of Kronecker products of 2x2 spin
matrices, and Hubbard Hamiltonians through the Jordan-Wigner transformation:
no bit strings, ranks or popcount signs are used.  Sector projections select
basis states with plain Python loops.

Conventions (stated in the oracle): site i <-> binary digit i of the state
index, digit 1 = up spin / occupied orbital.  Fermion modes: up orbital of
site i is mode i, down orbital is mode N + i; a Fock state is
prod_{m ascending, occupied} c^+_m |0>, so c^+_m = Z_0 ... Z_{m-1} a^+_m.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp

SZ = np.array([[-0.5, 0.0], [0.0, 0.5]])   # local basis (down, up)
SP = np.array([[0.0, 0.0], [1.0, 0.0]])    # S^+ |down> = |up>
SM = SP.T.copy()
ZF = np.array([[1.0, 0.0], [0.0, -1.0]])    # (-1)^n on (empty, occupied)
AD = np.array([[0.0, 0.0], [1.0, 0.0]])     # a^+ |0> = |1>
I2 = np.eye(2)


def site_op(op, i, n):
    """op on digit i of an n-digit index (digit i has weight 2^i)."""
    mats = [I2] * n
    mats[n - 1 - i] = op           # leftmost factor = most significant digit
    out = sp.csr_matrix(np.array([[1.0]]))
    for m in mats:
        out = sp.kron(out, sp.csr_matrix(m), format="csr")
    return out


def spin_hamiltonian(n_sites, terms):
    """Sum over EXCHANGE / XXZ terms of Jz SzSz + Jxy (S+S- + S-S+)/2."""
    D = 1 << n_sites
    H = sp.csr_matrix((D, D))
    for kind, i, j, spin, v0, v1 in terms:
        Jz = v0
        Jxy = v0 if kind == "EXCHANGE" else v1
        H = H + Jz * site_op(SZ, i, n_sites) @ site_op(SZ, j, n_sites)
        H = H + 0.5 * Jxy * (site_op(SP, i, n_sites) @ site_op(SM, j, n_sites)
                             + site_op(SM, i, n_sites) @ site_op(SP, j, n_sites))
    return H.tocsr()


def fermion_cdag(m, n_modes):
    mats = []
    for k in range(n_modes - 1, -1, -1):   # leftmost = mode n_modes-1
        mats.append(ZF if k < m else (AD if k == m else I2))
    out = sp.csr_matrix(np.array([[1.0]]))
    for a in mats:
        out = sp.kron(out, sp.csr_matrix(a), format="csr")
    return out


def hubbard_hamiltonian(n_sites, terms):
    M = 2 * n_sites
    cd = [fermion_cdag(m, M) for m in range(M)]
    c = [x.T.tocsr() for x in cd]
    num = [cd[m] @ c[m] for m in range(M)]
    D = 1 << M
    H = sp.csr_matrix((D, D))
    for kind, i, j, spin, v0, v1 in terms:
        if kind == "HOP":
            for s in ((0, 1) if spin == -1 else (spin,)):
                a, b = i + s * n_sites, j + s * n_sites
                H = H - v0 * (cd[a] @ c[b] + cd[b] @ c[a])
        elif kind == "HUBBARD_U":
            H = H + v0 * (num[i] @ num[i + n_sites])
        elif kind == "DENS_DENS":
            ni = num[i] + num[i + n_sites]
            nj = num[j] + num[j + n_sites]
            H = H + v0 * (ni @ nj)
    return H.tocsr()


def strings_with_popcount(n_bits, k):
    return sorted(sum(1 << p for p in c) for c in itertools.combinations(range(n_bits), k))


def spin_sector_indices(n_sites, n_up):
    return np.array(strings_with_popcount(n_sites, n_up), dtype=np.int64)


def hubbard_sector_indices(n_sites, n_up, n_dn):
    ups = strings_with_popcount(n_sites, n_up)
    dns = strings_with_popcount(n_sites, n_dn)
    return np.array([su | (sd << n_sites) for su in ups for sd in dns], dtype=np.int64)


def project(H, idx):
    return H[idx][:, idx].toarray()
