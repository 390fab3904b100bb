"""Circuit-text parser for the noisy circuit model of Sec. 2 (oracle side).

Test infrastructure only.  The grammar is Stim-like (the paper's benchmark
circuits are Stim-style text with DETECTOR / OBSERVABLE_INCLUDE and R_Z / R_X,
Sec. 7) and covers the operation families of Sec. 2:

  Clifford gates      I H S S_DAG SQRT_X SQRT_X_DAG X Y Z CX CNOT CY CZ SWAP
  Pauli rotations     R_X(t) R_Y(t) R_Z(t) T T_DAG R_PAULI(t) <product>
                      with R_P(t) = exp(-i t P / 2)
  Pauli measurements  M MX MY MR MRX R RX MPP <product>...
  Pauli noise         X_ERROR(p) Y_ERROR(p) Z_ERROR(p) DEPOLARIZE1(p)
                      DEPOLARIZE2(p) PAULI_CHANNEL_1(px,py,pz)
  feedback            CX|CY|CZ rec[-k] q  (Pauli on q if the record bit is 1)
  annotations         DETECTOR rec[..]..  OBSERVABLE_INCLUDE(i) rec[..]..
                      TICK QUBIT_COORDS SHIFT_COORDS (ignored), REPEAT n { }

Resets follow the paper's model (Sec. 2: Pauli measurements plus
record-controlled Pauli feedback): R q is a hidden (unrecorded) Z measurement
followed by X^m on q, RX a hidden X measurement followed by Z^m, MR / MRX the
recorded measurement followed by the same feedback.

Output: a flat list of operations after REPEAT unrolling, each measurement
carrying its ordinal t (all measurement events, recorded or hidden) and each
noise location its channel ordinal c, both in circuit order.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import re

PAULI_CHARS = "IXYZ"


@dataclass
class Op:
    kind: str                 # clifford | rot | meas | fb | noise | det | obs
    name: str = ""
    qubits: tuple = ()
    pauli: tuple = ()         # ((q, 'X'|'Y'|'Z'), ...) sorted by q
    theta: float = 0.0
    t: int = -1               # measurement ordinal
    rec: int = -1             # record index (-1: hidden)
    conds: tuple = ()         # measurement ordinals whose parity controls fb / det / obs
    c: int = -1               # noise channel ordinal
    q: float = 0.0            # noise: total error probability
    cells: tuple = ()         # noise: tuple of paulis
    weights: tuple = ()       # noise: cell weights
    index: int = -1           # det / obs index


@dataclass
class Circuit:
    ops: list = field(default_factory=list)
    num_qubits: int = 0
    num_meas: int = 0          # measurement ordinals
    num_records: int = 0
    num_channels: int = 0
    num_dets: int = 0
    num_obs: int = 0
    record_ordinal: list = field(default_factory=list)   # record index -> t


class ParseError(ValueError):
    pass


_ONE_Q = {"I", "H", "S", "S_DAG", "SQRT_X", "SQRT_X_DAG", "X", "Y", "Z"}
_TWO_Q = {"CX": "CX", "CNOT": "CX", "CY": "CY", "CZ": "CZ", "SWAP": "SWAP"}
_IGNORED = {"TICK", "QUBIT_COORDS", "SHIFT_COORDS"}

_D2_CELLS = []
for _a in range(4):
    for _b in range(4):
        if _a == 0 and _b == 0:
            continue
        _D2_CELLS.append((_a, _b))


def _parse_product(tok: str):
    out = {}
    for part in tok.split("*"):
        m = re.fullmatch(r"([XYZ])(\d+)", part)
        if not m:
            raise ParseError(f"bad Pauli product term {part!r}")
        q = int(m.group(2))
        if q in out:
            raise ParseError(f"repeated qubit {q} in product {tok!r}")
        out[q] = m.group(1)
    return tuple(sorted(out.items()))


class _Builder:
    def __init__(self):
        self.c = Circuit()
        self.max_q = -1

    def qubit(self, tok):
        if not re.fullmatch(r"\d+", tok):
            raise ParseError(f"bad qubit target {tok!r}")
        q = int(tok)
        self.max_q = max(self.max_q, q)
        return q

    def rec_ordinal(self, tok):
        m = re.fullmatch(r"rec\[-(\d+)\]", tok)
        if not m:
            raise ParseError(f"bad record target {tok!r}")
        k = int(m.group(1))
        if k < 1 or k > self.c.num_records:
            raise ParseError(f"record {tok} out of range")
        return self.c.record_ordinal[self.c.num_records - k]

    def meas(self, pauli, recorded):
        for q, _ in pauli:
            self.max_q = max(self.max_q, q)
        t = self.c.num_meas
        self.c.num_meas += 1
        rec = -1
        if recorded:
            rec = self.c.num_records
            self.c.num_records += 1
            self.c.record_ordinal.append(t)
        self.c.ops.append(Op("meas", pauli=pauli, t=t, rec=rec))
        return t

    def noise(self, qubits, q, cells, weights):
        c = self.c.num_channels
        self.c.num_channels += 1
        self.c.ops.append(Op("noise", qubits=tuple(qubits), c=c, q=q,
                             cells=tuple(cells), weights=tuple(weights)))


def _split_args(name_tok):
    m = re.fullmatch(r"([A-Z_0-9]+)(?:\(([^)]*)\))?", name_tok)
    if not m:
        raise ParseError(f"bad instruction {name_tok!r}")
    args = []
    if m.group(2) is not None and m.group(2).strip() != "":
        for a in m.group(2).split(","):
            args.append(float(a))
    return m.group(1), args


def _lines(text):
    out = []
    for raw in text.splitlines():
        line = raw.split("#", 1)[0].strip()
        if line:
            out.append(line)
    return out


def _exec_lines(b: _Builder, lines):
    pos = 0
    while pos < len(lines):
        line = lines[pos]
        toks = line.split()
        if line == "}":
            raise ParseError("unmatched }")
        if toks[0] == "REPEAT":
            if len(toks) != 3 or toks[2] != "{" or not re.fullmatch(r"\d+", toks[1]):
                raise ParseError(f"bad REPEAT line {line!r}")
            n = int(toks[1])
            depth = 1
            j = pos + 1
            while j < len(lines):
                if lines[j].split()[0] == "REPEAT":
                    depth += 1
                elif lines[j] == "}":
                    depth -= 1
                    if depth == 0:
                        break
                j += 1
            if j >= len(lines):
                raise ParseError("unterminated REPEAT")
            body = lines[pos + 1:j]
            for _ in range(n):
                _exec_lines(b, body)
            pos = j + 1
            continue
        name, args = _split_args(toks[0])
        _exec_instr(b, name, args, toks[1:])
        pos += 1


def _exec_instr(b: _Builder, name, args, targets):
    c = b.c
    if name in _IGNORED:
        return
    if name in _ONE_Q:
        if args:
            raise ParseError(f"{name} takes no arguments")
        for tok in targets:
            q = b.qubit(tok)
            c.ops.append(Op("clifford", name=name, qubits=(q,)))
        return
    if name in _TWO_Q:
        g = _TWO_Q[name]
        if len(targets) % 2:
            raise ParseError(f"{name} needs target pairs")
        for i in range(0, len(targets), 2):
            a, bb = targets[i], targets[i + 1]
            a_rec, b_rec = a.startswith("rec"), bb.startswith("rec")
            if a_rec and b_rec:
                raise ParseError("feedback between two records")
            if a_rec or b_rec:
                if g == "SWAP":
                    raise ParseError("SWAP cannot be record-controlled")
                if b_rec and g != "CZ":
                    raise ParseError(f"{g} target cannot be a record")
                rt, qt = (a, bb) if a_rec else (bb, a)
                t = b.rec_ordinal(rt)
                q = b.qubit(qt)
                p = {"CX": "X", "CY": "Y", "CZ": "Z"}[g]
                c.ops.append(Op("fb", pauli=((q, p),), conds=(t,)))
                continue
            qa, qb = b.qubit(a), b.qubit(bb)
            if qa == qb:
                raise ParseError(f"{name} on identical qubits")
            c.ops.append(Op("clifford", name=g, qubits=(qa, qb)))
        return
    if name in ("R_X", "R_Y", "R_Z", "T", "T_DAG"):
        if name in ("T", "T_DAG"):
            if args:
                raise ParseError(f"{name} takes no arguments")
            theta = (3.141592653589793 / 4.0) * (1.0 if name == "T" else -1.0)
            axis = "Z"
        else:
            if len(args) != 1:
                raise ParseError(f"{name} needs one angle")
            theta = args[0]
            axis = name[2]
        for tok in targets:
            q = b.qubit(tok)
            c.ops.append(Op("rot", pauli=((q, axis),), theta=theta))
        return
    if name == "R_PAULI":
        if len(args) != 1:
            raise ParseError("R_PAULI needs one angle")
        for tok in targets:
            p = _parse_product(tok)
            for q, _ in p:
                b.max_q = max(b.max_q, q)
            c.ops.append(Op("rot", pauli=p, theta=args[0]))
        return
    if name in ("M", "MX", "MY", "MR", "MRX", "R", "RX"):
        if args:
            raise ParseError(f"{name} takes no arguments")
        axis = {"M": "Z", "MR": "Z", "R": "Z", "MX": "X", "MRX": "X", "RX": "X", "MY": "Y"}[name]
        for tok in targets:
            q = b.qubit(tok)
            recorded = name not in ("R", "RX")
            t = b.meas(((q, axis),), recorded)
            if name in ("MR", "MRX", "R", "RX"):
                fbp = "X" if axis == "Z" else "Z"
                c.ops.append(Op("fb", pauli=((q, fbp),), conds=(t,)))
        return
    if name == "MPP":
        if args:
            raise ParseError("MPP takes no arguments")
        for tok in targets:
            b.meas(_parse_product(tok), True)
        return
    if name in ("X_ERROR", "Y_ERROR", "Z_ERROR", "DEPOLARIZE1", "PAULI_CHANNEL_1"):
        if name == "PAULI_CHANNEL_1":
            if len(args) != 3:
                raise ParseError("PAULI_CHANNEL_1 needs 3 probabilities")
            px, py, pz = args
            qtot = (px + py) + pz
            cells = [("X",), ("Y",), ("Z",)]
            weights = [px, py, pz]
        else:
            if len(args) != 1:
                raise ParseError(f"{name} needs one probability")
            qtot = args[0]
            if name == "DEPOLARIZE1":
                cells = [("X",), ("Y",), ("Z",)]
                weights = [1.0, 1.0, 1.0]
            else:
                cells = [(name[0],)]
                weights = [1.0]
        if not (0.0 <= qtot <= 1.0):
            raise ParseError(f"{name} probability out of range")
        for tok in targets:
            q = b.qubit(tok)
            b.noise((q,), qtot, [tuple((q, ch) for ch in cell) for cell in cells], weights)
        return
    if name == "DEPOLARIZE2":
        if len(args) != 1:
            raise ParseError("DEPOLARIZE2 needs one probability")
        if not (0.0 <= args[0] <= 1.0):
            raise ParseError("DEPOLARIZE2 probability out of range")
        if len(targets) % 2:
            raise ParseError("DEPOLARIZE2 needs target pairs")
        for i in range(0, len(targets), 2):
            qa, qb = b.qubit(targets[i]), b.qubit(targets[i + 1])
            if qa == qb:
                raise ParseError("DEPOLARIZE2 on identical qubits")
            cells = []
            for pa, pb in _D2_CELLS:
                cell = []
                if pa:
                    cell.append((qa, PAULI_CHARS[pa]))
                if pb:
                    cell.append((qb, PAULI_CHARS[pb]))
                cells.append(tuple(cell))
            b.noise((qa, qb), args[0], cells, [1.0] * 15)
        return
    if name == "DETECTOR":
        conds = tuple(b.rec_ordinal(tok) for tok in targets)
        c.ops.append(Op("det", conds=conds, index=c.num_dets))
        c.num_dets += 1
        return
    if name == "OBSERVABLE_INCLUDE":
        if len(args) != 1 or args[0] != int(args[0]) or args[0] < 0:
            raise ParseError("OBSERVABLE_INCLUDE needs a non-negative index")
        k = int(args[0])
        conds = tuple(b.rec_ordinal(tok) for tok in targets)
        c.ops.append(Op("obs", conds=conds, index=k))
        c.num_obs = max(c.num_obs, k + 1)
        return
    raise ParseError(f"unsupported instruction {name!r}")


def parse(text: str) -> Circuit:
    b = _Builder()
    lines = _lines(text)
    _exec_lines(b, lines)
    b.c.num_qubits = b.max_q + 1
    return b.c
