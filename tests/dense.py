"""Dense 2^n matrix checks for small n (test infrastructure).

Everything here is built from the textbook 2x2 Pauli matrices with np.kron
(qubit 0 is the leftmost factor), independently of the oracle's letter table
and of the CUDA library's bit formulas.
"""
import numpy as np

PAULI = {
    "I": np.eye(2, dtype=complex),
    "X": np.array([[0, 1], [1, 0]], dtype=complex),
    "Y": np.array([[0, -1j], [1j, 0]], dtype=complex),
    "Z": np.array([[1, 0], [0, -1]], dtype=complex),
}


def letters(n, xrow, zrow):
    out = []
    for j in range(n):
        xb = (int(xrow[j // 64]) >> (j % 64)) & 1
        zb = (int(zrow[j // 64]) >> (j % 64)) & 1
        out.append("IXYZ"[(1 if xb and not zb else 2 if xb and zb else 3 if zb else 0)])
    return "".join(out)


def bits(word, W):
    """'XIZY' -> (x[W], z[W]) as uint64 arrays."""
    x = np.zeros(W, np.uint64)
    z = np.zeros(W, np.uint64)
    for j, l in enumerate(word):
        if l in "XY":
            x[j // 64] |= np.uint64(1 << (j % 64))
        if l in "ZY":
            z[j // 64] |= np.uint64(1 << (j % 64))
    return x, z


def pauli_matrix(word):
    m = np.ones((1, 1), dtype=complex)
    for l in word:
        m = np.kron(m, PAULI[l])
    return m


def dense(n, x, z, c):
    H = np.zeros((2 ** n, 2 ** n), dtype=complex)
    for i in range(len(c)):
        H += c[i] * pauli_matrix(letters(n, x[i], z[i]))
    return H


def qmf_state(theta, phi):
    """Eq. 3 product state, qubit 0 leftmost."""
    v = np.ones(1, dtype=complex)
    for t, p in zip(theta, phi):
        v = np.kron(v, np.array([np.cos(t / 2), np.exp(1j * p) * np.sin(t / 2)]))
    return v


def conjugate(Hm, word, tau):
    """e^{-i tau P/2} H e^{+i tau P/2}, with e^{-i tau P/2} = cos(tau/2) I - i sin(tau/2) P."""
    P = pauli_matrix(word)
    U = np.cos(tau / 2) * np.eye(len(P)) - 1j * np.sin(tau / 2) * P
    return U @ Hm @ U.conj().T


def expval(Hm, psi):
    return np.vdot(psi, Hm @ psi)


def decompose_coefficient(Hm, word):
    """Tr(P H) / 2^n."""
    return np.trace(pauli_matrix(word) @ Hm) / Hm.shape[0]
