import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: long CPU test")


def load_golden(name):
    """Parse a tests/golden/*.txt fixture: 'key: numbers' lines, '#' comments."""
    import numpy as np
    out = {}
    with open(os.path.join(ROOT, "tests", "golden", name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            k, v = line.split(":", 1)
            out[k.strip()] = np.array([float(t) for t in v.split()])
    return out


def parity_scale(model, want, mu_ref=1.0):
    """Per-variable normalisation for GPU-vs-oracle errors.

    Each conserved variable is compared relative to the natural size of the
    terms that make it up, not to its own maximum when that is a cancellation:
      - vector components share one scale (max over the three components);
      - S = rho h W^2 v + E x B (Eq. resistive prims): the scale of S includes
        max |E| |B|, since the two parts cancel in near-static magnetised states;
      - two fluids: Dbar, Sbar, taubar are sums of mu_s-weighted species terms
        (Eq. twoFluid cons), so their scale is mu_ref times that of D, S, tau;
      - varrho, psi, phi (charge and divergence-cleaning fields, Sec. 2.1.1)
        start at round-off size and are scaled by the field magnitude max(|E|, |B|).
    """
    import numpy as np
    m = np.abs(want).reshape(want.shape[0], -1).max(axis=1)
    s = m.copy()
    bs, es = (5, 8) if model == 0 else (10, 13)
    B, E = want[bs:bs + 3], want[es:es + 3]
    # S = rho h W^2 v + E x B (Eq. resistive prims): its natural size includes |E| |B|
    exb = float(np.max(np.sqrt((B * B).sum(axis=0) * (E * E).sum(axis=0))))
    if model == 0:
        groups = [(1, 4), (5, 8), (8, 11)]
        for a, b in groups:
            s[a:b] = m[a:b].max()
        s[1:4] = max(s[1], exb)
        em = max(s[5], s[8])
        for v in (11, 12, 13):
            s[v] = max(m[v], em)
    else:
        for a, b in [(1, 4), (6, 9), (10, 13), (13, 16)]:
            s[a:b] = m[a:b].max()
        s[1:4] = max(s[1], exb)
        s[5] = max(m[5], mu_ref * m[0])
        s[6:9] = max(s[6], mu_ref * s[1])
        s[9] = max(m[9], mu_ref * m[4])
        em = max(s[10], s[13])
        for v in (16, 17):
            s[v] = max(m[v], em)
    return np.maximum(s, 1e-300)


def parity_errors(model, got, want, mu_ref=1.0):
    """max |got - want| per variable divided by parity_scale."""
    import numpy as np
    d = np.abs(got - want).reshape(want.shape[0], -1).max(axis=1)
    return d / parity_scale(model, want, mu_ref)
