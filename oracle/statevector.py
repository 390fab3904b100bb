"""Dense FP64 state-vector sampler: the ground truth for small circuits.

Test infrastructure only.  It simulates the noisy circuit model of Sec. 2
literally, one shot at a time, with no factorization and no planning:

  * Clifford gates multiply the state by their 2x2 / 4x4 matrices,
  * R_P(theta) = cos(theta/2) I - i sin(theta/2) P,
  * a Pauli measurement of P computes p0 = || (I + P)/2 psi ||^2, takes the
    recorded bit from the shared stream rule (0 iff u < p0), projects with
    (I + (-1)^m P)/2 and renormalises,
  * noise applies the Pauli cell the shared noise stream selected,
  * feedback applies its Pauli when the parity of the named outcomes is 1.

Qubit q is bit q of the amplitude index.  It is also the exact reference for
record distributions: ``exact_distribution`` enumerates every measurement
branch (and every noise cell of the listed channels) with its probability.
Pins (tests/test_oracle_sv.py): closed forms (cos^2(pi/8) after H; R_Z(pi/4);
MX, Pr(1) = p for X_ERROR(p); M, ...), agreement with the tableau sampler on
random Clifford circuits shot by shot, and probability conservation.
"""
from __future__ import annotations

import numpy as np

from .noise import NoiseSampler
from .records import POSTSELECT_NONE, finalize
from .streams import meas_uniform, outcome_from

_SQ2 = 1.0 / np.sqrt(2.0)
_GATES1 = {
    "I": np.eye(2, dtype=complex),
    "H": np.array([[1, 1], [1, -1]], dtype=complex) * _SQ2,
    "S": np.array([[1, 0], [0, 1j]], dtype=complex),
    "S_DAG": np.array([[1, 0], [0, -1j]], dtype=complex),
    "X": np.array([[0, 1], [1, 0]], dtype=complex),
    "Y": np.array([[0, -1j], [1j, 0]], dtype=complex),
    "Z": np.array([[1, 0], [0, -1]], dtype=complex),
    "SQRT_X": 0.5 * np.array([[1 + 1j, 1 - 1j], [1 - 1j, 1 + 1j]], dtype=complex),
    "SQRT_X_DAG": 0.5 * np.array([[1 - 1j, 1 + 1j], [1 + 1j, 1 - 1j]], dtype=complex),
}


def _controlled(u):
    m = np.eye(4, dtype=complex)
    m[2:, 2:] = u
    return m


# two-qubit matrices in the basis |a b> with a the first (control) qubit as MSB
_GATES2 = {
    "CX": _controlled(_GATES1["X"]),
    "CY": _controlled(_GATES1["Y"]),
    "CZ": _controlled(_GATES1["Z"]),
    "SWAP": np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]], dtype=complex),
}


class StateVector:
    def __init__(self, n: int):
        if n > 24:
            raise ValueError("state-vector oracle limited to 24 qubits")
        self.n = n
        self.psi = np.zeros(1 << n, dtype=np.complex128)
        self.psi[0] = 1.0
        self._idx = np.arange(1 << n, dtype=np.int64)

    def _tensor(self):
        # axis i of the reshaped tensor is qubit n-1-i
        return self.psi.reshape((2,) * self.n)

    def apply1(self, u, q):
        t = self._tensor()
        ax = self.n - 1 - q
        t = np.moveaxis(np.tensordot(u, t, axes=([1], [ax])), 0, ax)
        self.psi = np.ascontiguousarray(t).reshape(-1)

    def apply2(self, u, qa, qb):
        t = self._tensor()
        axa, axb = self.n - 1 - qa, self.n - 1 - qb
        u4 = u.reshape(2, 2, 2, 2)
        t = np.tensordot(u4, t, axes=([2, 3], [axa, axb]))
        t = np.moveaxis(t, [0, 1], [axa, axb])
        self.psi = np.ascontiguousarray(t).reshape(-1)

    def pauli_apply(self, pauli, vec=None):
        """Return P @ vec (vec defaults to the state)."""
        v = self.psi if vec is None else vec
        flip = 0
        phase = np.ones(1 << self.n, dtype=np.complex128)
        for q, ch in pauli:
            bit = (self._idx >> q) & 1
            if ch == "X":
                flip |= 1 << q
            elif ch == "Z":
                phase *= np.where(bit == 1, -1.0, 1.0)
            elif ch == "Y":
                flip |= 1 << q
                # Y|0> = i|1>, Y|1> = -i|0>:  factor on the source basis state
                phase *= np.where(bit == 1, -1j, 1j)
        out = np.empty_like(v)
        out[self._idx ^ flip] = phase * v
        return out

    def gate(self, name, qubits):
        if len(qubits) == 1:
            self.apply1(_GATES1[name], qubits[0])
        else:
            self.apply2(_GATES2[name], qubits[0], qubits[1])

    def rotate(self, pauli, theta):
        self.psi = np.cos(theta / 2) * self.psi - 1j * np.sin(theta / 2) * self.pauli_apply(pauli)

    def branch_probability(self, pauli):
        ppsi = self.pauli_apply(pauli)
        phi0 = 0.5 * (self.psi + ppsi)
        return float(np.vdot(phi0, phi0).real), ppsi

    def project(self, pauli, m, ppsi=None):
        if ppsi is None:
            ppsi = self.pauli_apply(pauli)
        sgn = 1.0 if m == 0 else -1.0
        phi = 0.5 * (self.psi + sgn * ppsi)
        pm = float(np.vdot(phi, phi).real)
        if pm <= 1e-300:
            raise FloatingPointError("projection onto a zero-probability branch")
        self.psi = phi / np.sqrt(pm)
        return pm


def sample_shot(circuit, seed: int, r: int, noise: NoiseSampler | None = None,
                prob_log: list | None = None):
    """Simulate shot r; returns the list of outcomes indexed by ordinal."""
    if noise is None:
        noise = NoiseSampler(circuit, seed)
    fired = noise.shot(r)
    sv = StateVector(circuit.num_qubits)
    out = [0] * circuit.num_meas
    for op in circuit.ops:
        k = op.kind
        if k == "clifford":
            sv.gate(op.name, op.qubits)
        elif k == "rot":
            sv.rotate(op.pauli, op.theta)
        elif k == "noise":
            cell = fired.get(op.c)
            if cell is not None:
                sv.psi = sv.pauli_apply(op.cells[cell])
        elif k == "meas":
            p0, ppsi = sv.branch_probability(op.pauli)
            u = meas_uniform(seed, op.t, r)
            m = outcome_from(p0, u)
            if prob_log is not None:
                prob_log.append((op.t, p0))
            sv.project(op.pauli, m, ppsi)
            out[op.t] = m
        elif k == "fb":
            v = 0
            for t in op.conds:
                v ^= out[t]
            if v:
                sv.psi = sv.pauli_apply(op.pauli)
    return out


def sample(circuit, seed: int, shots, postselect: int = POSTSELECT_NONE, post_dets=None):
    """Sample the listed shot indices (iterable of ints).

    Returns dict of uint8 arrays: records (S, R), dets (S, D), obs (S, O),
    discard (S,), outcomes (S, num_meas).
    """
    shots = list(shots)
    noise = NoiseSampler(circuit, seed)
    recs, dets, obss, disc, outs = [], [], [], [], []
    for r in shots:
        o = sample_shot(circuit, seed, r, noise)
        rec, det, obs, d = finalize(circuit, o, postselect, post_dets)
        recs.append(rec)
        dets.append(det)
        obss.append(obs)
        disc.append(d)
        outs.append(o)
    S = len(shots)
    return {
        "records": np.array(recs, dtype=np.uint8).reshape(S, circuit.num_records),
        "dets": np.array(dets, dtype=np.uint8).reshape(S, circuit.num_dets),
        "obs": np.array(obss, dtype=np.uint8).reshape(S, circuit.num_obs),
        "discard": np.array(disc, dtype=np.uint8),
        "outcomes": np.array(outs, dtype=np.uint8).reshape(S, circuit.num_meas),
    }


def exact_distribution(circuit, noise_free: bool = False, max_branches: int = 1 << 16):
    """Exact distribution of the record bit-string.

    Enumerates every noise cell of every channel (unless noise_free) and every
    measurement branch.  Returns {records tuple: probability}.  Intended for
    tiny circuits only.
    """
    n = circuit.num_qubits
    dist = {}
    count = [0]

    def rec_tuple(out):
        return tuple(out[t] for t in circuit.record_ordinal)

    def walk(i, psi, out, prob):
        count[0] += 1
        if count[0] > max_branches:
            raise RuntimeError("too many branches")
        sv = StateVector(n)
        sv.psi = psi
        while i < len(circuit.ops):
            op = circuit.ops[i]
            k = op.kind
            if k == "clifford":
                sv.gate(op.name, op.qubits)
            elif k == "rot":
                sv.rotate(op.pauli, op.theta)
            elif k == "noise":
                if noise_free or op.q == 0.0:
                    i += 1
                    continue
                tot = sum(op.weights)
                walk(i + 1, sv.psi.copy(), list(out), prob * (1.0 - op.q))
                for cell, w in zip(op.cells, op.weights):
                    if w == 0.0:
                        continue
                    walk(i + 1, sv.pauli_apply(cell), list(out), prob * op.q * w / tot)
                return
            elif k == "meas":
                p0, ppsi = sv.branch_probability(op.pauli)
                for m, pm in ((0, p0), (1, 1.0 - p0)):
                    if pm < 1e-14:
                        continue
                    s2 = StateVector(n)
                    s2.psi = sv.psi.copy()
                    s2.project(op.pauli, m, ppsi)
                    o2 = list(out)
                    o2[op.t] = m
                    walk(i + 1, s2.psi, o2, prob * pm)
                return
            elif k == "fb":
                v = 0
                for t in op.conds:
                    v ^= out[t]
                if v:
                    sv.psi = sv.pauli_apply(op.pauli)
            i += 1
        key = rec_tuple(out)
        dist[key] = dist.get(key, 0.0) + prob

    init = np.zeros(1 << n, dtype=np.complex128)
    init[0] = 1.0
    walk(0, init, [0] * circuit.num_meas, 1.0)
    return dist
