"""CPU oracle for the SymFT per-shot sampling engine (test infrastructure only).

This package is the plain, slow, independent reference that the CUDA sampler is
checked against.  Only the test suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it; the
product path never does.  It shares no code with ``paper_2607_28600_b300``:
its own circuit parser, its own Philox, its own simulators.

Modules
-------
philox      Philox4x32-10 block function (Salmon et al., SC'11), numpy.
streams     the shared random-stream specification (noise blocks, measurement
            uniforms) written from its definition.
circuit     parser of the Stim-like circuit text of the noisy circuit model
            (Sec. 2) into a flat operation list with channel / measurement
            ordinals.
statevector dense FP64 state-vector sampler (ground truth, small n).
tableau     Aaronson-Gottesman stabilizer tableau sampler (ground truth for
            pure-Clifford circuits of any size).
symft       plain FP64 SymFT: frame factorization (Sec. 3), stabilizer-
            coordinate planning (Sec. 4) and the single-shot sampler (Sec. 5),
            one shot at a time, unpacked bits.
records     detector / observable parities and the postselection rule.

Parity status: every function here is pinned by tests under ``tests/`` marked
``not gpu`` (closed forms, brute force, library outputs); see each module's
header for the pins that apply to it.
"""
