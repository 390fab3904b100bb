"""Seeded synthetic circuit generators (inputs only; no sampling arithmetic).

The paper's benchmark circuits live in an external repository that is not
available here, so every workload is generated from a seed with the shapes of
the paper's workloads (Sec. 7): rotated surface-code memory (Sec. 7.2:
d=7,r=7 has 97 qubits and 336 detectors, d=9,r=9 has 161 qubits and 720
detectors), surface-code memory with coherent over-rotations, a
cultivation-shaped near-Clifford circuit, 15-to-1 distillation and random
near-Clifford circuits.  Each generator returns circuit text in the
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


def coherent_surface_code_memory(d: int, rounds: int, p: float = 1e-3, eps: float = 0.02) -> str:
    """Rotated surface-code Z memory with coherent over-rotations: after every
    CX layer, R_Z(eps) = exp(-i eps Z / 2) on both qubits of each CX, on top of
    the circuit-level noise of `rotated_surface_code_memory`.

    This is the shape of the paper's coherent-noise workload (Sec. 7: a small
    R_Z(0.02) over-rotation with circuit-level noise on distance-d surface-code
    circuits over r rounds).  Its peak active width grows with d and r: 4, 8,
    12 and 24 for (d, r) = (3, 1), (3, 3), (5, 1), (5, 5).
    """
    out = []
    for line in rotated_surface_code_memory(d, rounds, p).splitlines():
        out.append(line)
        if line.startswith("CX "):
            out.append(f"R_Z({eps!r}) " + " ".join(line.split()[1:]))
    return "\n".join(out) + "\n"


# ---------------------------------------------------------------------------
# [[15,1,3]] quantum Reed-Muller code and 15-to-1 distillation
# ---------------------------------------------------------------------------

def _rref_pivots(rows):
    """Reduced row echelon form over GF(2); returns (rows, pivot columns)."""
    rows = [list(r) for r in rows]
    n = len(rows[0])
    piv = []
    r = 0
    for col in range(n):
        sel = None
        for i in range(r, len(rows)):
            if rows[i][col]:
                sel = i
                break
        if sel is None:
            continue
        rows[r], rows[sel] = rows[sel], rows[r]
        for i in range(len(rows)):
            if i != r and rows[i][col]:
                rows[i] = [a ^ b for a, b in zip(rows[i], rows[r])]
        piv.append(col)
        r += 1
        if r == len(rows):
            break
    return rows, piv


def reed_muller_15_encoder():
    """CSS encoder of the [[15,1,3]] code (qubit v-1 <-> nonzero v in F_2^4).

    X stabilizers: X on {v : v_i = 1}, i = 0..3; logical X = X on all 15.
    Returns (stab_pivots, logical_pivot, cnots) such that: logical state on
    logical_pivot, |+> on stab_pivots, |0> elsewhere, then the CNOTs (control,
    target) in order, gives the encoded state.  The logical row (all-ones word
    reduced against the stabilizer rows, so it is zero on their pivots) is
    spread first; the stabilizer rows, which may cover the logical pivot,
    follow.
    """
    gx = [[(v >> i) & 1 for v in range(1, 16)] for i in range(4)]
    rows, piv = _rref_pivots(gx)
    logical = [1] * 15
    for r, p in zip(rows, piv):
        if logical[p]:
            logical = [a ^ b for a, b in zip(logical, r)]
    lp = logical.index(1)
    cnots = [(lp, j) for j in range(15) if j != lp and logical[j]]
    for r, p in zip(rows, piv):
        cnots += [(p, j) for j in range(15) if j != p and r[j]]
    return piv, lp, cnots


def distillation_15_to_1(p: float = 1e-3, variant: str = "literal") -> str:
    """15-to-1 T-state distillation on 16 qubits (15 code qubits + output 15).

    literal: 15 qubits in |+>, DEPOLARIZE1(p) then R_Z(pi/4) = exp(-i pi/8 Z)
             on each, the Reed-Muller decoder (inverse encoder), 14 mid-circuit
             Z measurements (detectors on the four X-type syndromes, the only
             deterministic ones for ideal inputs), the logical moved to qubit
             15 with record-controlled Z feedback, output measured in X.
    encoded: |+_L> encoded first, then the noisy rotations (transversal T on
             the encoded state), then the same decoder / measurement stage.
    """
    stab_piv, log_piv, cnots = reed_muller_15_encoder()
    e = _Emitter(p)
    qs = list(range(15))
    e.reset(qs + [15])
    if variant == "encoded":
        e.g1("H", sorted(stab_piv + [log_piv]))
        for c in cnots:              # sequential: the two row groups do not commute
            e.cx([c])
    elif variant == "literal":
        e.g1("H", qs)
    else:
        raise ValueError(variant)
    e.raw(f"DEPOLARIZE1({p!r}) " + " ".join(map(str, qs)) if p > 0 else "TICK")
    e.raw(f"R_Z({PI / 4!r}) " + " ".join(map(str, qs)))
    # decoder: inverse encoder
    for c in reversed(cnots):
        e.cx([c])
    e.g1("H", sorted(stab_piv))
    syn = [q for q in qs if q != log_piv]
    base = e.nrec
    e.measure(syn, "Z")
    rec = {q: base + i for i, q in enumerate(syn)}
    # literal: only the X-type syndromes (stabilizer pivots) are deterministic
    # for ideal T|+> inputs; the encoded variant checks all fourteen
    for q in (syn if variant == "encoded" else sorted(stab_piv)):
        e.raw(f"DETECTOR rec[-{e.nrec - rec[q]}]")
    # move the logical to the output qubit, with record-controlled Z feedback
    e.cx([(log_piv, 15)])
    e.cx([(15, log_piv)])
    for q in stab_piv:
        e.raw(f"CZ rec[-{e.nrec - rec[q]}] 15")
    e.g1("H", [15])
    e.measure([15], "Z")
    e.raw("OBSERVABLE_INCLUDE(0) rec[-1]")
    return e.text()


# ---------------------------------------------------------------------------
# cultivation-shaped circuit: d=3 color code, T-check layer, growth to d=9
# ---------------------------------------------------------------------------

COLOR_CODE_D3 = [(0, 1, 2, 3), (1, 2, 4, 5), (2, 3, 5, 6)]   # Steane plaquettes


def cultivation_shaped(p: float = 1e-3, grow_d: int = 9, grow_rounds: int = 3,
                       check_layers: int = 2, stage: str = "full") -> str:
    """Cultivation-shaped near-Clifford circuit.

    1. d=3 color code (7 data qubits 0..6), logical |+> prepared by measuring
       the Z plaquettes of |+>^7, two rounds of X / Z plaquette checks (MPP),
       detectors comparing rounds;
    2. `check_layers` transversal check layers: exp(+i pi/8 Z) on each data
       qubit, a logical X check (MPP X^7) and the plaquette checks, then
       exp(-i pi/8 Z) on each data qubit; detectors on deterministic checks;
    3. (stage "full") growth to a d=`grow_d` rotated surface code whose first
       data qubits are the color-code qubits, `grow_rounds` rounds of its
       stabilizer checks, detectors between consecutive grown rounds.
    Noise: DEPOLARIZE1(p) on the data before every check, X_ERROR/Z_ERROR on
    MPP results via DEPOLARIZE1 on the measured qubits.  Every detector is a
    candidate for postselection.
    """
    e = _Emitter(p)
    data = list(range(7))
    e.reset(data)
    e.g1("H", data)

    def checks(prev):
        cur = {}
        for kind in ("X", "Z"):
            for i, pl in enumerate(COLOR_CODE_D3):
                if p > 0:
                    e.raw(f"DEPOLARIZE1({p!r}) " + " ".join(map(str, pl)))
                e.raw("MPP " + "*".join(f"{kind}{q}" for q in pl))
                e.nrec += 1
                cur[(kind, i)] = e.nrec - 1
                if prev is not None and (kind, i) in prev:
                    e.raw(f"DETECTOR rec[-1] rec[-{e.nrec - prev[(kind, i)]}]")
        return cur

    # round 0 fixes the random Z plaquettes; rounds 1..2 compare to it
    prev = checks(None)
    for _ in range(2):
        prev = checks(prev)
    for _ in range(check_layers):
        e.raw(f"R_Z({PI / 4!r}) " + " ".join(map(str, data)))
        if p > 0:
            e.raw(f"DEPOLARIZE1({p!r}) " + " ".join(map(str, data)))
        e.raw("MPP " + "*".join(f"X{q}" for q in data))
        e.nrec += 1
        prev = checks(prev)
        e.raw(f"R_Z({-PI / 4!r}) " + " ".join(map(str, data)))
    if stage != "full":
        base = e.nrec
        e.measure(data, "X")
        e.raw("OBSERVABLE_INCLUDE(0) " + " ".join(f"rec[-{e.nrec - (base + i)}]" for i in range(7)))
        return e.text()
    # growth: a d=grow_d rotated surface code whose data qubits 0..6 are the
    # color-code qubits; the other data qubits start in |0>
    d = grow_d
    plaqs = rotated_surface_code_layout(d)
    new_data = list(range(7, d * d))
    e.reset(new_data)
    ancs = [a for _, _, a in plaqs]
    xanc = [a for t, _, a in plaqs if t == "X"]
    e.reset(ancs)
    anc_rec = None
    for rnd in range(grow_rounds):
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
        if anc_rec is not None:
            for _, _, a in plaqs:
                e.raw(f"DETECTOR rec[-{e.nrec - cur[a]}] rec[-{e.nrec - anc_rec[a]}]")
        anc_rec = cur
    base = e.nrec
    dq = list(range(d * d))
    e.measure(dq, "Z")
    e.raw("OBSERVABLE_INCLUDE(0) " + " ".join(f"rec[-{e.nrec - (base + c)}]" for c in range(d)))
    return e.text()


def mixed_batch(seed: int = 1, n: int = 64, p: float = 1e-3):
    """Mixed workload: `n` circuits drawn from a seed.

    Surface-code memory (d = 3..11, d rounds), cultivation-shaped circuits
    (growth to d = 5 or 9), 15-to-1 distillation (encoded / literal) and random
    near-Clifford circuits on 20..100 qubits with 0..24 rotations of uniform
    random angle on weight-1..4 Paulis.  Returns [(name, text, postselect)].
    """
    rng = random.Random(seed)
    out = []
    for i in range(n):
        kind = rng.choices(["surface", "cultivation", "distill", "random"], [0.3, 0.15, 0.15, 0.4])[0]
        if kind == "surface":
            d = rng.choice([3, 5, 7, 9, 11])
            out.append((f"surface_d{d}_{i}", rotated_surface_code_memory(d, d, p), 0))
        elif kind == "cultivation":
            g = rng.choice([5, 9])
            out.append((f"cultivation_g{g}_{i}", cultivation_shaped(p, grow_d=g), 1))
        elif kind == "distill":
            v = rng.choice(["encoded", "literal"])
            out.append((f"distill_{v}_{i}", distillation_15_to_1(p, v), 1))
        else:
            nq = rng.randint(20, 100)
            nr = rng.randint(0, 24)
            out.append((f"random_n{nq}_r{nr}_{i}",
                        random_near_clifford(nq, rng.randint(8, 30), nr, p=p, seed=rng.randrange(1 << 30)), 0))
    return out
