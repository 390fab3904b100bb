"""Random circuit text for tests (seeded; generators only)."""


def random_clifford_text(rng, n, depth, noise=True, rot=0.0, feedback=True):
    lines = []
    g1 = ["H", "S", "S_DAG", "SQRT_X", "SQRT_X_DAG", "X", "Y", "Z"]
    g2 = ["CX", "CY", "CZ", "SWAP"]
    nrec = 0
    for _ in range(depth):
        if rot and rng.random() < rot:
            k = rng.randint(1, min(3, n))
            qs = rng.sample(range(n), k)
            th = rng.uniform(-3, 3)
            if k == 1 and rng.random() < 0.5:
                lines.append(f"{rng.choice(['R_X', 'R_Y', 'R_Z'])}({th!r}) {qs[0]}")
            else:
                lines.append(f"R_PAULI({th!r}) " + "*".join(f"{rng.choice('XYZ')}{q}" for q in qs))
            continue
        r = rng.random()
        if r < 0.35:
            lines.append(f"{rng.choice(g1)} {rng.randrange(n)}")
        elif r < 0.6:
            a, b = rng.sample(range(n), 2)
            lines.append(f"{rng.choice(g2)} {a} {b}")
        elif r < 0.75:
            k = rng.randint(1, min(3, n))
            qs = rng.sample(range(n), k)
            lines.append("MPP " + "*".join(f"{rng.choice('XYZ')}{q}" for q in qs))
            nrec += 1
        elif r < 0.8:
            lines.append(f"{rng.choice(['M', 'MX', 'MY', 'MR', 'MRX'])} {rng.randrange(n)}")
            nrec += 1
        elif r < 0.85:
            lines.append(f"{rng.choice(['R', 'RX'])} {rng.randrange(n)}")
        elif r < 0.9 and nrec > 0 and feedback:
            lines.append(f"{rng.choice(['CX', 'CY', 'CZ'])} rec[-{rng.randint(1, nrec)}] {rng.randrange(n)}")
        elif noise:
            if rng.random() < 0.5:
                lines.append(f"DEPOLARIZE1(0.2) {rng.randrange(n)}")
            else:
                a, b = rng.sample(range(n), 2)
                lines.append(f"DEPOLARIZE2(0.3) {a} {b}")
    lines.append("M " + " ".join(str(q) for q in range(n)))
    nrec += n
    # a few detectors / observables over random records
    for i in range(3):
        k = rng.randint(1, min(3, nrec))
        recs = sorted(rng.sample(range(1, nrec + 1), k))
        lines.append("DETECTOR " + " ".join(f"rec[-{x}]" for x in recs))
    lines.append(f"OBSERVABLE_INCLUDE(0) rec[-1] rec[-{min(2, nrec)}]")
    return "\n".join(lines) + "\n"


def fusion_circuit_text(rng, n=6, blocks=6, noise_p=0.05):
    """Random circuit with rewrite opportunities for the commutation-aware
    simplification: a rotation R_P, then operations on other qubits (and
    sometimes noise, a feedback or a measurement on P's support, which make
    the two signs differ by a symbol or make the operations anticommute), then
    a second rotation of the same Pauli P, at times with the opposite angle
    (cancellation), at times followed by a measurement of P (branch phase)."""
    lines = [f"H {q}" for q in range(n)]
    for q in range(n):
        if rng.random() < 0.5:
            lines.append(f"S {q}")
    nrec = 0
    for _ in range(blocks):
        k = rng.randint(1, 2)
        sup = rng.sample(range(n), k)
        pstr = "*".join(f"{rng.choice('XYZ')}{q}" for q in sup)
        th = rng.uniform(-2.5, 2.5)
        lines.append(f"R_PAULI({th!r}) {pstr}")
        others = [q for q in range(n) if q not in sup]
        for _ in range(rng.randint(0, 3)):
            r = rng.random()
            if r < 0.3 and len(others) >= 2:
                a, b = rng.sample(others, 2)
                lines.append(f"CX {a} {b}")
            elif r < 0.5 and others:
                lines.append(f"R_Z({rng.uniform(-1, 1)!r}) {rng.choice(others)}")
            elif r < 0.65 and others:
                lines.append(f"DEPOLARIZE1({noise_p}) {rng.choice(others)}")
            elif r < 0.75:
                lines.append(f"DEPOLARIZE1({noise_p}) {rng.choice(sup)}")
            elif r < 0.85 and others:
                lines.append(f"M {rng.choice(others)}")
                nrec += 1
            elif nrec:
                lines.append(f"CZ rec[-1] {rng.choice(sup)}")
        r = rng.random()
        if r < 0.4:
            lines.append(f"R_PAULI({-th!r}) {pstr}")
        elif r < 0.7:
            lines.append(f"R_PAULI({rng.uniform(-2, 2)!r}) {pstr}")
        if rng.random() < 0.3:
            lines.append(f"MPP {pstr}")
            nrec += 1
            lines.append("DETECTOR rec[-1]")
    lines.append("M " + " ".join(str(q) for q in range(n)))
    nrec += n
    lines.append(f"DETECTOR rec[-1] rec[-2]")
    lines.append("OBSERVABLE_INCLUDE(0) rec[-1]")
    return "\n".join(lines) + "\n"
