"""Aaronson-Gottesman stabilizer tableau sampler (ground truth for Clifford circuits).

Test infrastructure only.  S. Aaronson and D. Gottesman, "Improved simulation
of stabilizer circuits", PRA 70, 052328 (2004) -- the CHP algorithm the paper
cites for stabilizer simulation (Sec. 8).  Rows 0..n-1 are destabilizers,
rows n..2n-1 stabilizers, row 2n is scratch; a Pauli is (x, z) bits with
(1, 1) the Hermitian Y, plus a sign bit.

For a circuit without non-Clifford rotations the x/z part of the tableau
evolves identically in every shot (noise, feedback and measurement outcomes
only flip signs), so the sign column is held per shot: ``r`` has shape
(2n+1, S).  Per shot this is exactly the CHP algorithm:

  gates           AG's update rules (H, S, CX; the rest composed from them or,
                  for Pauli gates, as sign flips of anticommuting rows),
  measurement     of a Pauli P (generalised AG): random iff a stabilizer
                  anticommutes with P -- the outcome is then the shared-stream
                  bit (Pr = 1/2) and the tableau is updated by rowsum; else
                  the outcome is the sign of the product of the stabilizers
                  whose destabilizers anticommute with P,
  noise/feedback  applying Pauli Q flips the sign of every row that
                  anticommutes with Q.

Pins (tests/test_oracle_tableau.py): agreement with the state-vector sampler
shot by shot on random Clifford circuits, GHZ / Bell parity facts, and the
noiseless-QEC invariant (no detector fires).
"""
from __future__ import annotations

import numpy as np

from .noise import NoiseSampler
from .records import POSTSELECT_NONE, finalize
from .streams import mbit_words


def _g(x1, z1, x2, z2):
    """AG's phase exponent contribution of multiplying (x1,z1) into (x2,z2)."""
    x1 = x1.astype(np.int64)
    z1 = z1.astype(np.int64)
    x2 = x2.astype(np.int64)
    z2 = z2.astype(np.int64)
    out = np.zeros_like(x1)
    y = (x1 == 1) & (z1 == 1)
    xo = (x1 == 1) & (z1 == 0)
    zo = (x1 == 0) & (z1 == 1)
    out = np.where(y, z2 - x2, out)
    out = np.where(xo, z2 * (2 * x2 - 1), out)
    out = np.where(zo, x2 * (1 - 2 * z2), out)
    return out


class Tableau:
    def __init__(self, n: int, S: int):
        self.n = n
        self.S = S
        self.x = np.zeros((2 * n + 1, n), dtype=np.uint8)
        self.z = np.zeros((2 * n + 1, n), dtype=np.uint8)
        self.r = np.zeros((2 * n + 1, S), dtype=np.uint8)
        for i in range(n):
            self.x[i, i] = 1
            self.z[n + i, i] = 1

    # --- gates (AG update rules) -------------------------------------------------
    def h(self, a):
        self.r ^= (self.x[:, a] & self.z[:, a])[:, None]
        self.x[:, a], self.z[:, a] = self.z[:, a].copy(), self.x[:, a].copy()

    def s(self, a):
        self.r ^= (self.x[:, a] & self.z[:, a])[:, None]
        self.z[:, a] ^= self.x[:, a]

    def s_dag(self, a):
        self.r ^= (self.x[:, a] & (1 - self.z[:, a]))[:, None]
        self.z[:, a] ^= self.x[:, a]

    def cx(self, a, b):
        self.r ^= (self.x[:, a] & self.z[:, b] & (self.x[:, b] ^ self.z[:, a] ^ 1))[:, None]
        self.x[:, b] ^= self.x[:, a]
        self.z[:, a] ^= self.z[:, b]

    def gate(self, name, qs):
        if name == "I":
            return
        if name == "H":
            self.h(qs[0])
        elif name == "S":
            self.s(qs[0])
        elif name == "S_DAG":
            self.s_dag(qs[0])
        elif name == "SQRT_X":
            self.h(qs[0]); self.s(qs[0]); self.h(qs[0])
        elif name == "SQRT_X_DAG":
            self.h(qs[0]); self.s_dag(qs[0]); self.h(qs[0])
        elif name in ("X", "Y", "Z"):
            self.apply_pauli(((qs[0], name),), np.ones(self.S, dtype=np.uint8))
        elif name == "CX":
            self.cx(qs[0], qs[1])
        elif name == "CZ":
            self.h(qs[1]); self.cx(qs[0], qs[1]); self.h(qs[1])
        elif name == "CY":
            self.s_dag(qs[1]); self.cx(qs[0], qs[1]); self.s(qs[1])
        elif name == "SWAP":
            a, b = qs
            self.x[:, [a, b]] = self.x[:, [b, a]]
            self.z[:, [a, b]] = self.z[:, [b, a]]
        else:
            raise ValueError(name)

    # --- Pauli helpers -------------------------------------------------------------
    def pauli_bits(self, pauli):
        px = np.zeros(self.n, dtype=np.uint8)
        pz = np.zeros(self.n, dtype=np.uint8)
        for q, ch in pauli:
            if ch in ("X", "Y"):
                px[q] = 1
            if ch in ("Z", "Y"):
                pz[q] = 1
        return px, pz

    def anticommuting_rows(self, px, pz, rows):
        sym = (self.x[rows] @ pz.astype(np.int64) + self.z[rows] @ px.astype(np.int64)) & 1
        return np.asarray(rows)[sym == 1]

    def apply_pauli(self, pauli, mask):
        """Apply Pauli to the shots whose mask bit is 1 (sign flips)."""
        px, pz = self.pauli_bits(pauli)
        rows = self.anticommuting_rows(px, pz, np.arange(2 * self.n))
        if len(rows):
            self.r[rows] ^= mask[None, :]

    def rowsum(self, h, i):
        g = int(_g(self.x[i], self.z[i], self.x[h], self.z[h]).sum())
        g &= 3
        if g not in (0, 2):
            raise AssertionError("rowsum of anticommuting rows")
        self.r[h] ^= self.r[i]
        if g == 2:
            self.r[h] ^= 1
        self.x[h] ^= self.x[i]
        self.z[h] ^= self.z[i]

    def measure(self, pauli, random_bits):
        """Measure Pauli P on every shot; random_bits (S,) used if random.

        Returns (outcomes (S,) uint8, is_random bool).
        """
        n = self.n
        px, pz = self.pauli_bits(pauli)
        stab = self.anticommuting_rows(px, pz, np.arange(n, 2 * n))
        if len(stab):
            p = int(stab[0])
            anti = self.anticommuting_rows(px, pz, np.arange(2 * n))
            for i in anti:
                # the paired destabilizer p - n is overwritten just below
                if int(i) != p and int(i) != p - n:
                    self.rowsum(int(i), p)
            self.x[p - n] = self.x[p]
            self.z[p - n] = self.z[p]
            self.r[p - n] = self.r[p]
            self.x[p] = px
            self.z[p] = pz
            self.r[p] = random_bits
            return random_bits.copy(), True
        s = 2 * n
        self.x[s] = 0
        self.z[s] = 0
        self.r[s] = 0
        destab = self.anticommuting_rows(px, pz, np.arange(n))
        for i in destab:
            self.rowsum(s, int(i) + n)
        if not (np.array_equal(self.x[s], px) and np.array_equal(self.z[s], pz)):
            raise AssertionError("deterministic measurement did not reproduce P")
        return self.r[s].copy(), False


def _has_rotation(circuit):
    return any(op.kind == "rot" for op in circuit.ops)


def outcomes(circuit, seed: int, shots):
    """(S, num_meas) uint8 outcomes of the listed shots (any order)."""
    if _has_rotation(circuit):
        raise ValueError("tableau oracle handles Clifford circuits only")
    shots = np.asarray(list(shots), dtype=np.int64)
    S = len(shots)
    tab = Tableau(circuit.num_qubits, S)
    noise = NoiseSampler(circuit, seed)
    # per-shot noise: {channel: cell} for each shot
    fired = [noise.shot(int(r)) for r in shots]
    by_channel = {}
    for j, f in enumerate(fired):
        for c, cell in f.items():
            by_channel.setdefault(c, []).append((j, cell))
    out = np.zeros((S, circuit.num_meas), dtype=np.uint8)
    words = shots >> 6
    bits = shots & 63
    for op in circuit.ops:
        k = op.kind
        if k == "clifford":
            tab.gate(op.name, op.qubits)
        elif k == "noise":
            for j, cell in by_channel.get(op.c, ()):
                mask = np.zeros(S, dtype=np.uint8)
                mask[j] = 1
                tab.apply_pauli(op.cells[cell], mask)
        elif k == "meas":
            uw = sorted(set(int(w) for w in words))
            wmap = {}
            for w in uw:
                wmap[w] = int(mbit_words(seed, op.t, w, 1)[0])
            rb = np.array([(wmap[int(w)] >> int(b)) & 1 for w, b in zip(words, bits)],
                          dtype=np.uint8)
            m, _ = tab.measure(op.pauli, rb)
            out[:, op.t] = m
        elif k == "fb":
            v = np.zeros(S, dtype=np.uint8)
            for t in op.conds:
                v ^= out[:, t]
            if v.any():
                tab.apply_pauli(op.pauli, v)
        elif k in ("det", "obs"):
            pass
        else:
            raise ValueError(k)
    return out


def sample(circuit, seed: int, shots, postselect: int = POSTSELECT_NONE, post_dets=None):
    shots = list(shots)
    o = outcomes(circuit, seed, shots)
    recs, dets, obss, disc = [], [], [], []
    for j in range(len(shots)):
        rec, det, obs, d = finalize(circuit, o[j], postselect, post_dets)
        recs.append(rec)
        dets.append(det)
        obss.append(obs)
        disc.append(d)
    S = len(shots)
    return {
        "records": np.array(recs, dtype=np.uint8).reshape(S, circuit.num_records),
        "dets": np.array(dets, dtype=np.uint8).reshape(S, circuit.num_dets),
        "obs": np.array(obss, dtype=np.uint8).reshape(S, circuit.num_obs),
        "discard": np.array(disc, dtype=np.uint8),
        "outcomes": o,
    }
