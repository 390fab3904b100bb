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
