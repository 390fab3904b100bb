"""Plain FP64 SymFT: factorization, planning and single-shot sampling (oracle side).

Test infrastructure only.  A literal, one-shot-at-a-time restatement of the
method, kept in the paper's order and notation:

  Sec. 3  symbolic Clifford-Pauli frame factorization: the Clifford frame C_t
          (held as its pull-back map P -> C_t^dag P C_t), the symbolic Pauli
          frame E_t (one-hot noise variables s_{c,j}, Eq. symbolic-noise-sign;
          feedback terms), and the pulled-back rotations / projectors with
          their affine signs lambda (Eq. factorization-invariant).
  Sec. 4  stabilizer-coordinate planning over the stabilizer-destabilizer
          tableau (Zbar_j, Xbar_j), active width k, the decomposition
          P = mu Xbar_A^a Zbar_A^b Xbar_D^d Zbar_D^c (Eq. active-dormant-
          decomposition) and the seven instruction kinds: PromoteRot,
          ActiveDiagRot, ActivePairRot (Sec. 4.1); RandomMeas, DetMeas,
          ActiveDiagMeas, ActivePairMeas (Sec. 4.2), with the symbolic
          corrections of the measurement cases propagated to the suffix.
  Sec. 5  the single-shot algorithm: sample s and m1, walk the instructions,
          substitute lambda[nu], apply the dense updates, sample active
          outcomes, record.

Readings where the paper leaves a choice (the same ones the CUDA path takes):
  * active index: coordinate j (1-based) is bit j-1 of the amplitude index,
    a promoted coordinate becomes the most significant bit;
  * dormant pivot: the lowest dormant coordinate with d = 1, swapped to k+1;
  * active pivot: the highest set bit of a (pair) or of b (diagonal); the
    retired pivot pair becomes the first dormant coordinate;
  * measurement outcome: 0 iff u(t, r) < Pr(m_t = 0) (oracle.streams).

Pins (tests/test_oracle_symft.py): per-shot equality with the state-vector
sampler on random near-Clifford circuits, the closed forms of Sec. 4 cases,
k bookkeeping (k_final = #PromoteRot - #active measurements) and the norm
invariant after every measurement.
"""
from __future__ import annotations

import math

import numpy as np

from .noise import NoiseSampler
from .records import POSTSELECT_NONE, finalize
from .streams import mbit_word, meas_uniform, outcome_from

# ---------------------------------------------------------------------------
# Paulis: (x, z, e) = i^e X^x Z^z with x, z python-int bit masks over qubits.
# ---------------------------------------------------------------------------


def pmul(p1, p2):
    x1, z1, e1 = p1
    x2, z2, e2 = p2
    e = (e1 + e2 + 2 * ((z1 & x2).bit_count())) & 3
    return (x1 ^ x2, z1 ^ z2, e)


def omega(p1, p2):
    """Anticommutation indicator (Sec. 3)."""
    return ((p1[0] & p2[1]) ^ (p1[1] & p2[0])).bit_count() & 1


def from_chars(pauli):
    """Hermitian Pauli from ((q, 'X'|'Y'|'Z'), ...):  Y = i X Z."""
    x = z = e = 0
    for q, ch in pauli:
        if ch in ("X", "Y"):
            x |= 1 << q
        if ch in ("Z", "Y"):
            z |= 1 << q
        if ch == "Y":
            e += 1
    return (x, z, e & 3)


def is_hermitian(p):
    return (p[2] & 1) == ((p[0] & p[1]).bit_count() & 1)


# local gate conjugation tables g^dag Q g, computed from the matrices
_SQ2 = 1.0 / math.sqrt(2.0)
_M1 = {
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


def _ctl(u):
    m = np.eye(4, dtype=complex)
    m[2:, 2:] = u
    return m


_M2 = {  # basis |a b>, a = first target = most significant
    "CX": _ctl(_M1["X"]), "CY": _ctl(_M1["Y"]), "CZ": _ctl(_M1["Z"]),
    "SWAP": np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]], dtype=complex),
}
_P1 = {"X": _M1["X"], "Z": _M1["Z"]}


def _local_paulis(nq):
    """All (x, z, e) on nq local qubits with their matrices (local qubit 0 = first target)."""
    out = []
    for x in range(1 << nq):
        for z in range(1 << nq):
            m = np.eye(1, dtype=complex)
            for lq in range(nq):       # local qubit 0 is the most significant factor
                f = np.eye(2, dtype=complex)
                if (x >> lq) & 1:
                    f = f @ _M1["X"]
                if (z >> lq) & 1:
                    f = f @ _M1["Z"]
                m = np.kron(m, f)
            for e in range(4):
                out.append(((x, z, e), (1j ** e) * m))
    return out


_CONJ_CACHE = {}


def _conj_table(name):
    """g^dag Q g for Q in {X_0, Z_0, (X_1, Z_1)} as local (x, z, e)."""
    if name in _CONJ_CACHE:
        return _CONJ_CACHE[name]
    if name in _M1:
        g, nq = _M1[name], 1
    else:
        g, nq = _M2[name], 2
    cands = _local_paulis(nq)
    table = {}
    for lq in range(nq):
        for ch in ("X", "Z"):
            q = np.eye(1, dtype=complex)
            for j in range(nq):
                q = np.kron(q, _P1[ch] if j == lq else np.eye(2))
            target = g.conj().T @ q @ g
            hit = None
            for p, m in cands:
                if np.allclose(m, target):
                    hit = p
                    break
            assert hit is not None
            table[(lq, ch)] = hit
    _CONJ_CACHE[name] = table
    return table


# ---------------------------------------------------------------------------
# Sec. 3: factorization
# ---------------------------------------------------------------------------


class Expr:
    """Affine Boolean expression: constant bit + XOR of symbols (int bit mask)."""
    __slots__ = ("mask", "const")

    def __init__(self, mask=0, const=0):
        self.mask = mask
        self.const = const

    def __xor__(self, o):
        return Expr(self.mask ^ o.mask, self.const ^ o.const)

    def value(self, nu_mask):
        return ((self.mask & nu_mask).bit_count() & 1) ^ self.const


class Factorizer:
    """Maintains C_t (pull-back map), E_t (symbolic Pauli frame)."""

    def __init__(self, circuit):
        self.c = circuit
        n = circuit.num_qubits
        self.n = n
        self.TX = [(1 << q, 0, 0) for q in range(n)]    # C^dag X_q C
        self.TZ = [(0, 1 << q, 0) for q in range(n)]    # C^dag Z_q C
        # symbols: noise one-hot s_{c,j} first, then measurement ordinals
        self.noise_sym = {}
        nsym = 0
        for op in circuit.ops:
            if op.kind == "noise":
                for j in range(len(op.cells)):
                    self.noise_sym[(op.c, j)] = nsym
                    nsym += 1
        self.meas_base = nsym
        self.nsym = nsym + circuit.num_meas
        self.terms = []        # (Expr, Pauli) factors of E_t

    def msym(self, t):
        return self.meas_base + t

    def pull_back(self, p):
        """C^dag P C for P = (x, z, e) physical."""
        x, z, e = p
        out = (0, 0, e)
        q = 0
        xx = x
        while xx:
            if xx & 1:
                out = pmul(out, self.TX[q])
            xx >>= 1
            q += 1
        q = 0
        zz = z
        while zz:
            if zz & 1:
                out = pmul(out, self.TZ[q])
            zz >>= 1
            q += 1
        return out

    def clifford(self, name, qubits):
        tab = _conj_table(name)
        nq = len(qubits)
        newX, newZ = {}, {}
        for lq in range(nq):
            for ch in ("X", "Z"):
                lx, lz, le = tab[(lq, ch)]
                px = pz = 0
                for j in range(nq):
                    if (lx >> j) & 1:
                        px |= 1 << qubits[j]
                    if (lz >> j) & 1:
                        pz |= 1 << qubits[j]
                img = self.pull_back((px, pz, le))
                (newX if ch == "X" else newZ)[qubits[lq]] = img
        for q, v in newX.items():
            self.TX[q] = v
        for q, v in newZ.items():
            self.TZ[q] = v

    def sign(self, pp):
        """lambda with E^dag P' E = (-1)^lambda P' for pulled-back P'."""
        lam = Expr()
        for ex, q in self.terms:
            if omega(q, pp):
                lam = lam ^ ex
        return lam

    def add_term(self, ex, pulled_pauli):
        self.terms.append((ex, pulled_pauli))


# ---------------------------------------------------------------------------
# Sec. 4: planning
# ---------------------------------------------------------------------------


class Planner:
    def __init__(self, n):
        self.n = n
        self.Zb = [(0, 1 << j, 0) for j in range(n)]
        self.Xb = [(1 << j, 0, 0) for j in range(n)]
        self.k = 0

    def decompose(self, p):
        k, n = self.k, self.n
        a = b = 0
        d = []
        c = []
        for j in range(k):
            if omega(p, self.Zb[j]):
                a |= 1 << j
            if omega(p, self.Xb[j]):
                b |= 1 << j
        for j in range(k, n):
            d.append(omega(p, self.Zb[j]))
            c.append(omega(p, self.Xb[j]))
        q = (0, 0, 0)
        for j in range(k):
            if (a >> j) & 1:
                q = pmul(q, self.Xb[j])
        for j in range(k):
            if (b >> j) & 1:
                q = pmul(q, self.Zb[j])
        for j in range(k, n):
            if d[j - k]:
                q = pmul(q, self.Xb[j])
        for j in range(k, n):
            if c[j - k]:
                q = pmul(q, self.Zb[j])
        assert q[0] == p[0] and q[1] == p[1], "tableau does not span P"
        mu = (p[2] - q[2]) & 3     # P = i^mu Q
        return a, b, d, c, mu

    def _dormant_pivot_update(self, p, a, b, d, c):
        """Symplectic change with dormant pivot h (lowest with d=1); returns h."""
        k, n = self.k, self.n
        h = k + d.index(1)
        zh = self.Zb[h]
        for j in range(k):
            if (a >> j) & 1:
                self.Zb[j] = pmul(self.Zb[j], zh)
            if (b >> j) & 1:
                self.Xb[j] = pmul(self.Xb[j], zh)
        for j in range(k, n):
            if j == h:
                continue
            if d[j - k]:
                self.Zb[j] = pmul(self.Zb[j], zh)
            if c[j - k]:
                self.Xb[j] = pmul(self.Xb[j], zh)
        self.Xb[h] = p
        return h

    def _swap(self, i, j):
        self.Zb[i], self.Zb[j] = self.Zb[j], self.Zb[i]
        self.Xb[i], self.Xb[j] = self.Xb[j], self.Xb[i]

    def _retire_active(self, h):
        """Move active pair h to the dormant block (position k-1)."""
        zp, xp = self.Zb[h], self.Xb[h]
        for j in range(h, self.k - 1):
            self.Zb[j] = self.Zb[j + 1]
            self.Xb[j] = self.Xb[j + 1]
        self.Zb[self.k - 1] = zp
        self.Xb[self.k - 1] = xp
        self.k -= 1

    def rotation(self, p, theta, lam):
        a, b, d, c, mu = self.decompose(p)
        if any(d):
            self._dormant_pivot_update(p, a, b, d, c)
            h = self.k + d.index(1)
            if h != self.k:
                self._swap(h, self.k)
            self.k += 1
            return {"op": "PromoteRot", "theta": theta, "lam": lam}
        if a == 0 and b == 0:
            return None
        if a == 0:
            assert mu in (0, 2)
            return {"op": "ActiveDiagRot", "b": b, "mu": mu, "theta": theta, "lam": lam}
        return {"op": "ActivePairRot", "a": a, "b": b, "mu": mu, "theta": theta, "lam": lam}

    def measurement(self, p, t, lam):
        """Returns (instruction, correction Pauli or None, correction Expr)."""
        a, b, d, c, mu = self.decompose(p)
        k, n = self.k, self.n
        if any(d):
            h = self._dormant_pivot_update(p, a, b, d, c)
            zh = self.Zb[h]
            self.Zb[h], self.Xb[h] = p, zh          # Zbar'' = P, Xbar'' = Zbar_h
            corr = self.Xb[h]
            # correction exponent y_t = m_t xor lambda
            return {"op": "RandomMeas", "t": t}, corr, "m^lam"
        if a == 0 and b == 0:
            assert mu in (0, 2)
            return {"op": "DetMeas", "t": t, "eta": mu >> 1, "lam": lam}, None, None
        if a == 0:
            assert mu in (0, 2)
            eta = mu >> 1
            h = b.bit_length() - 1
            xh = self.Xb[h]
            for j in range(k):
                if j != h and (b >> j) & 1:
                    self.Xb[j] = pmul(self.Xb[j], xh)
            for j in range(k, n):
                if c[j - k]:
                    self.Xb[j] = pmul(self.Xb[j], xh)
            self.Zb[h] = (p[0], p[1], (p[2] + 2 * eta) & 3)    # (-1)^eta P
            corr = self.Xb[h]
            self._retire_active(h)
            return ({"op": "ActiveDiagMeas", "t": t, "b": b, "h": h, "eta": eta, "lam": lam},
                    corr, "m^lam^eta")
        h = a.bit_length() - 1
        zh = self.Zb[h]
        for j in range(k):
            if j == h:
                continue
            if (a >> j) & 1:
                self.Zb[j] = pmul(self.Zb[j], zh)
            if (b >> j) & 1:
                self.Xb[j] = pmul(self.Xb[j], zh)
        for j in range(k, n):
            if c[j - k]:
                self.Xb[j] = pmul(self.Xb[j], zh)
        self.Zb[h] = p
        self.Xb[h] = zh
        corr = self.Xb[h]
        self._retire_active(h)
        return ({"op": "ActivePairMeas", "t": t, "a": a, "b": b, "h": h, "mu": mu, "lam": lam},
                corr, "m^lam")


def compile_plan(circuit):
    """Factorize and plan; returns (instructions, factorizer, stats)."""
    f = Factorizer(circuit)
    pl = Planner(circuit.num_qubits)
    instrs = []
    kmax = 0
    for op in circuit.ops:
        kd = op.kind
        if kd == "clifford":
            f.clifford(op.name, op.qubits)
        elif kd == "noise":
            for j, cell in enumerate(op.cells):
                f.add_term(Expr(1 << f.noise_sym[(op.c, j)]), f.pull_back(from_chars(cell)))
        elif kd == "fb":
            ex = Expr()
            for t in op.conds:
                ex = ex ^ Expr(1 << f.msym(t))
            f.add_term(ex, f.pull_back(from_chars(op.pauli)))
        elif kd == "rot":
            pp = f.pull_back(from_chars(op.pauli))
            lam = f.sign(pp)
            ins = pl.rotation(pp, op.theta, lam)
            if ins is not None:
                instrs.append(ins)
        elif kd == "meas":
            pp = f.pull_back(from_chars(op.pauli))
            lam = f.sign(pp)
            ins, corr, how = pl.measurement(pp, op.t, lam)
            instrs.append(ins)
            if corr is not None:
                ex = Expr(1 << f.msym(op.t)) ^ lam
                if how == "m^lam^eta":
                    ex = ex ^ Expr(0, ins["eta"])
                f.add_term(ex, corr)
        kmax = max(kmax, pl.k)
    hist = {}
    for ins in instrs:
        hist[ins["op"]] = hist.get(ins["op"], 0) + 1
    return instrs, f, {"k_max": kmax, "k_final": pl.k, "hist": hist}


# ---------------------------------------------------------------------------
# Sec. 5: single-shot sampling
# ---------------------------------------------------------------------------


def _parity_vec(v):
    """Parity of each entry of an integer array."""
    return (np.bitwise_count(v) & 1).astype(np.int64)


def _insert_bit_vec(z, h, delta):
    """_insert_bit over an array of z."""
    low = z & ((1 << h) - 1)
    return low | (delta << h) | ((z >> h) << (h + 1))


def _insert_bit(z, h, delta):
    low = z & ((1 << h) - 1)
    return low | (delta << h) | ((z >> h) << (h + 1))


def _parity(v):
    return v.bit_count() & 1


class Plan:
    def __init__(self, circuit):
        self.circuit = circuit
        self.instrs, self.fact, self.stats = compile_plan(circuit)


def sample_shot(plan: Plan, seed: int, r: int, noise: NoiseSampler, prob_log=None,
                norm_log=None):
    """Outcomes (by ordinal) of shot r, following the single-shot algorithm."""
    c = plan.circuit
    f = plan.fact
    nu = 0
    # step 1: independent symbols -- noise s and the random measurement bits m1
    for ch, cell in noise.shot(r).items():
        nu |= 1 << f.noise_sym[(ch, cell)]
    for ins in plan.instrs:
        if ins["op"] == "RandomMeas":
            t = ins["t"]
            if (mbit_word(seed, t, r >> 6) >> (r & 63)) & 1:
                nu |= 1 << f.msym(t)
    out = [0] * c.num_meas
    alpha = np.ones(1, dtype=np.complex128)
    k = 0
    # steps 2-5: traverse the instruction stream
    for ins in plan.instrs:
        op = ins["op"]
        if op == "RandomMeas":
            t = ins["t"]
            out[t] = (nu >> f.msym(t)) & 1
            continue
        lam = ins["lam"].value(nu)
        if op == "DetMeas":
            m = lam ^ ins["eta"]
        elif op == "PromoteRot":
            th = ins["theta"]
            sgn = -1.0 if lam else 1.0
            alpha = np.concatenate([math.cos(th / 2) * alpha,
                                    -1j * sgn * math.sin(th / 2) * alpha])
            k += 1
            continue
        elif op == "ActiveDiagRot":
            th = ins["theta"]
            mu = 1.0 if ins["mu"] == 0 else -1.0
            sgn = -1.0 if lam else 1.0
            x = np.arange(1 << k, dtype=np.int64)
            par = _parity_vec(x & ins["b"])
            ang = -sgn * th * mu * np.where(par == 1, -1.0, 1.0) / 2.0
            alpha = np.exp(1j * ang) * alpha
            continue
        elif op == "ActivePairRot":
            # alpha'_x = cos(th/2) alpha_x - i sgn sin(th/2) mu (-1)^{b.(x^a)} alpha_{x^a}
            th = ins["theta"]
            mu = 1j ** ins["mu"]
            sgn = -1.0 if lam else 1.0
            a, b = ins["a"], ins["b"]
            x = np.arange(1 << k, dtype=np.int64)
            xa = x ^ a
            ph = np.where(_parity_vec(xa & b) == 1, -1.0, 1.0)
            alpha = (math.cos(th / 2) * alpha
                     - 1j * sgn * math.sin(th / 2) * mu * ph * alpha[xa])
            continue
        elif op == "ActiveDiagMeas":
            b, h, eta = ins["b"], ins["h"], ins["eta"]

            def branch(delta):
                # alpha at x(b, u(z, delta)): bit h of u(z, delta) corrected
                # by the parity of b over the other bits
                u = _insert_bit_vec(np.arange(1 << (k - 1), dtype=np.int64), h, delta)
                return alpha[u ^ (_parity_vec(u & ~(1 << h) & b) << h)]
            v0 = branch(0 ^ lam ^ eta)
            p0 = float(np.vdot(v0, v0).real)
            t = ins["t"]
            m = outcome_from(p0, meas_uniform(seed, t, r))
            if prob_log is not None:
                prob_log.append((t, p0))
            v = branch(m ^ lam ^ eta)
            pm = p0 if m == 0 else float(np.vdot(v, v).real)
            alpha = v / math.sqrt(pm)
            k -= 1
        elif op == "ActivePairMeas":
            a, b, h = ins["a"], ins["b"], ins["h"]
            muc = np.conj(1j ** ins["mu"])

            def beta(y):
                # beta_z(y) = (alpha_{u0} + conj(mu) (-1)^{b.u0 + y} alpha_{u0^a}) / sqrt(2)
                u0 = _insert_bit_vec(np.arange(1 << (k - 1), dtype=np.int64), h, 0)
                ph = np.where((_parity_vec(b & u0) ^ y) == 1, -1.0, 1.0)
                return (alpha[u0] + muc * ph * alpha[u0 ^ a]) / math.sqrt(2.0)
            v0 = beta(0 ^ lam)
            p0 = float(np.vdot(v0, v0).real)
            t = ins["t"]
            m = outcome_from(p0, meas_uniform(seed, t, r))
            if prob_log is not None:
                prob_log.append((t, p0))
            v = beta(m ^ lam)
            pm = p0 if m == 0 else float(np.vdot(v, v).real)
            alpha = v / math.sqrt(pm)
            k -= 1
        else:
            raise ValueError(op)
        t = ins["t"]
        out[t] = m
        if m:
            nu |= 1 << f.msym(t)
        if norm_log is not None:
            norm_log.append(float(np.vdot(alpha, alpha).real))
    return out


def sample(circuit, seed: int, shots, postselect: int = POSTSELECT_NONE, plan: Plan | None = None,
           prob_log=None, post_dets=None):
    if plan is None:
        plan = Plan(circuit)
    shots = list(shots)
    noise = NoiseSampler(circuit, seed)
    recs, dets, obss, disc, outs = [], [], [], [], []
    for r in shots:
        o = sample_shot(plan, seed, r, noise, prob_log=prob_log)
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
