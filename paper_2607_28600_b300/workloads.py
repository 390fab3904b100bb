"""Seeded synthetic circuit generators (inputs only; no sampling arithmetic).

The paper's benchmark circuits live in an external repository that is not
available here, so every workload is generated from a seed with the shapes of
the paper's workloads (Sec. 7): rotated surface-code memory (Sec. 7.2:
d=7,r=7 has 97 qubits and 336 detectors, d=9,r=9 has 161 qubits and 720
detectors), a cultivation-shaped near-Clifford circuit, 15-to-1 distillation
and random near-Clifford circuits.  Each generator returns circuit text in the
Stim-like grammar accepted by ``symft_compile``.

Noise model (the paper does not print one for its circuits): DEPOLARIZE1(p)
after every single-qubit Clifford and every reset, DEPOLARIZE2(p) after every
two-qubit Clifford, X_ERROR(p) (or Z_ERROR(p) for X-basis) immediately before
every measurement.
"""
from __future__ import annotations

import math
import random

PI = math.pi


class _Emitter:
    def __init__(self, p: float):
        self.p = float(p)
        self.lines: list[str] = []
        self.nrec = 0

    def raw(self, s):
        self.lines.append(s)

    def g1(self, name, qs):
        if not qs:
            return
        self.lines.append(f"{name} " + " ".join(map(str, qs)))
        if self.p > 0 and name != "I":
            self.lines.append(f"DEPOLARIZE1({self.p!r}) " + " ".join(map(str, qs)))

    def cx(self, pairs):
        if not pairs:
            return
        flat = [q for pr in pairs for q in pr]
        self.lines.append("CX " + " ".join(map(str, flat)))
        if self.p > 0:
            self.lines.append(f"DEPOLARIZE2({self.p!r}) " + " ".join(map(str, flat)))

    def reset(self, qs, basis="Z"):
        if not qs:
            return
        self.lines.append(("R " if basis == "Z" else "RX ") + " ".join(map(str, qs)))
        if self.p > 0:
            self.lines.append(f"DEPOLARIZE1({self.p!r}) " + " ".join(map(str, qs)))

    def measure(self, qs, basis="Z", reset=False):
        if not qs:
            return
        if self.p > 0:
            err = "X_ERROR" if basis == "Z" else "Z_ERROR"
            self.lines.append(f"{err}({self.p!r}) " + " ".join(map(str, qs)))
        op = {"Z": "M", "X": "MX"}[basis]
        if reset:
            op = {"Z": "MR", "X": "MRX"}[basis]
        self.lines.append(f"{op} " + " ".join(map(str, qs)))
        self.nrec += len(qs)
        if reset and self.p > 0:
            self.lines.append(f"DEPOLARIZE1({self.p!r}) " + " ".join(map(str, qs)))

    def text(self):
        return "\n".join(self.lines) + "\n"


def rotated_surface_code_layout(d: int):
    """Data qubits (r, c) -> r*d + c; plaquettes as (type, [data...] in CX order, ancilla).

    X plaquettes use the NW, NE, SW, SE order and Z plaquettes NW, SW, NE, SE
    (the N-order schedule that keeps hook errors perpendicular to the logical).
    """
    plaqs = []
    anc = d * d
    for r in range(-1, d):
        for c in range(-1, d):
            typ = "X" if (r + c) % 2 == 0 else "Z"
            cells = {}
            for dr, dc in ((0, 0), (0, 1), (1, 0), (1, 1)):
                rr, cc = r + dr, c + dc
                if 0 <= rr < d and 0 <= cc < d:
                    cells[(dr, dc)] = rr * d + cc
            if len(cells) == 4:
                keep = True
            elif len(cells) == 2:
                if typ == "X":
                    keep = (r == -1 or r == d - 1) and 0 <= c <= d - 2
                else:
                    keep = (c == -1 or c == d - 1) and 0 <= r <= d - 2
            else:
                keep = False
            if not keep:
                continue
            order = [(0, 0), (0, 1), (1, 0), (1, 1)] if typ == "X" else \
                    [(0, 0), (1, 0), (0, 1), (1, 1)]
            plaqs.append((typ, [cells.get(o) for o in order], anc))
            anc += 1
    return plaqs


def rotated_surface_code_memory(d: int, rounds: int, p: float = 1e-3,
                                t_on_data0_after_round: int | None = None,
                                t_angle: float = PI / 4) -> str:
    """Z-basis rotated surface-code memory, `rounds` rounds (0-indexed).

    With t_on_data0_after_round = r0, one R_Z(t_angle) = exp(-i t_angle Z / 2)
    acts on data qubit 0 right after round r0 (round r0 + 1 then sees it).
    """
    if d < 2 or rounds < 1:
        raise ValueError("need d >= 2 and rounds >= 1")
    plaqs = rotated_surface_code_layout(d)
    data = list(range(d * d))
    ancs = [a for _, _, a in plaqs]
    xanc = [a for t, _, a in plaqs if t == "X"]
    zplaq = [(ds, a) for t, ds, a in plaqs if t == "Z"]
    e = _Emitter(p)
    e.reset(data + ancs)
    anc_rec = {}      # ancilla -> record index of its latest measurement
    for rnd in range(rounds):
        e.raw("TICK")
        e.g1("H", xanc)
        for layer in range(4):
            pairs = []
            for typ, ds, a in plaqs:
                dq = ds[layer]
                if dq is None:
                    continue
                pairs.append((a, dq) if typ == "X" else (dq, a))
            e.cx(pairs)
        e.g1("H", xanc)
        base = e.nrec
        e.measure(ancs, "Z", reset=True)
        cur = {a: base + i for i, a in enumerate(ancs)}
        for typ, _, a in plaqs:
            if rnd == 0:
                if typ == "Z":
                    e.raw(f"DETECTOR rec[-{e.nrec - cur[a]}]")
            else:
                e.raw(f"DETECTOR rec[-{e.nrec - cur[a]}] rec[-{e.nrec - anc_rec[a]}]")
        anc_rec = cur
        if t_on_data0_after_round is not None and rnd == t_on_data0_after_round:
            e.raw(f"R_Z({t_angle!r}) 0")
    base = e.nrec
    e.measure(data, "Z")
    drec = {q: base + i for i, q in enumerate(data)}
    for ds, a in zplaq:
        targets = [f"rec[-{e.nrec - drec[q]}]" for q in ds if q is not None]
        targets.append(f"rec[-{e.nrec - anc_rec[a]}]")
        e.raw("DETECTOR " + " ".join(targets))
    e.raw("OBSERVABLE_INCLUDE(0) " + " ".join(f"rec[-{e.nrec - drec[c]}]" for c in range(d)))
    return e.text()


def random_near_clifford(n: int, layers: int, n_rot: int, p: float = 1e-3,
                         seed: int = 0, max_weight: int = 4) -> str:
    """Random H/S/CX layers with n_rot Pauli rotations of uniform random angle
    on random weight-1..max_weight Paulis, circuit noise p, final Z measurement."""
    rng = random.Random(seed)
    e = _Emitter(p)
    slots = sorted(rng.sample(range(layers), min(n_rot, layers))) if n_rot <= layers else \
        sorted(rng.randrange(layers) for _ in range(n_rot))
    rot_at = {}
    for s in slots:
        rot_at[s] = rot_at.get(s, 0) + 1
    for layer in range(layers):
        qs = list(range(n))
        rng.shuffle(qs)
        ones = {"H": [], "S": []}
        for q in qs[: n // 2]:
            ones[rng.choice(["H", "S"])].append(q)
        e.g1("H", sorted(ones["H"]))
        e.g1("S", sorted(ones["S"]))
        rest = qs[n // 2:]
        pairs = [(rest[i], rest[i + 1]) for i in range(0, len(rest) - 1, 2)]
        e.cx(pairs)
        for _ in range(rot_at.get(layer, 0)):
            w = rng.randint(1, min(max_weight, n))
            sup = rng.sample(range(n), w)
            th = rng.uniform(-PI, PI)
            prod = "*".join(f"{rng.choice('XYZ')}{q}" for q in sorted(sup))
            e.raw(f"R_PAULI({th!r}) {prod}")
    e.measure(list(range(n)), "Z")
    return e.text()
