"""Helpers of the full-size GPU tests: read the solver state a context saves
(aj_get_state) and check one GPU iteration against one oracle iteration taken
from the GPU's own x^T, x^{T-1} and beta_T, with the restart decision of
Algorithm alg-apg-re at T+1 taken on the oracle's d (rounding-level ties
either way)."""
import numpy as np

import oracle

HEADER = 64
STATE_BYTES = 152


def state_parts(blob, n):
    """One right-hand side: t, beta, K_ell, K_re and the iterates x^t, x^{t-1}
    (header: magic, n, nrhs, policy, state bytes, ...; then the RhsState; then
    the three iterate buffers)."""
    nrhs = int(np.frombuffer(blob[16:20], np.int32)[0])
    sbytes = int(np.frombuffer(blob[24:28], np.int32)[0])
    assert nrhs == 1 and sbytes == STATE_BYTES
    st = blob[HEADER:HEADER + sbytes]
    beta = float(np.frombuffer(st[8:16], np.float64)[0])
    t, ell, K, Kre = (int(v) for v in np.frombuffer(st[48:80], np.int64))
    cur, prev = (int(v) for v in np.frombuffer(st[88:96], np.int32))
    off = HEADER + sbytes
    bufs = [np.frombuffer(blob[off + k * 8 * n: off + (k + 1) * 8 * n], np.float64) for k in range(3)]
    return dict(t=t, beta=beta, K=K, Kre=Kre, x=bufs[cur], xprev=bufs[prev])


def one_step(Q, b, J, st, restarted):
    """The oracle's x^{T+1} from the GPU's state, and whether the GPU's
    decision at T+1 (``restarted``) is the rule's up to a rounding-level tie."""
    xT, xTm1 = st["x"], st["xprev"]
    T = st["t"]
    y = xT + st["beta"] * (xT - xTm1)
    cand = oracle.solve(Q, b, J, restart=False, maxit=1, stop=oracle.STOP_NONE, x0=y)["x"]
    g = oracle.spmv(Q, y) - b
    dx = cand - xT
    d = float(g @ dx)
    natural = (T + 1) > st["Kre"] + st["K"] and d >= 0.0
    if restarted != natural:
        assert abs(d) <= 1e-12 * np.linalg.norm(g) * np.linalg.norm(dx), (d, restarted)
    return xT if restarted else cand  # a restart at T+1 keeps x^{T+1} = x^T
