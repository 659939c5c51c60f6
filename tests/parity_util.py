"""Face-by-face parity protocol of npweno_reconstruct against the FP64 oracle.

1. Decisions.  The ENO stencil choice is the same arithmetic on both sides (FP64 path), or
   certified equal to it (mixed path), so the ENO bits are compared on every face.  The monotone
   switch is evaluated in closed form on the GPU and by a 4x4 elimination in the oracle; the two
   may differ only where a deciding quantity sits within the tie margin.  The switch bits are
   compared on every face that neither side marks as a switch near tie (oracle FLAG_SWITCH_TIE,
   GPU bit 1), and the share of such faces is bounded by the caller.
2. Replay.  The oracle is re-run with the GPU's flag stream as its switch and ENO decisions, and
   then every face value (v^-, v^+), every used shape parameter (FP64 path) and every guard /
   bound zeroing is compared on every face, ties included.
"""
import numpy as np

import oracle as O

GPU_NEAR_TIE = 0x02
GPU_ZERO_GUARD = 0x40
GPU_ZERO_BOUND = 0x80


def masks(k: int):
    """(switch bits, ENO bits) of the flag byte for k = 3 / k = 2."""
    if k == 2:
        return O.FLAG_SWITCH | O.FLAG_SWITCH_R_K2, 0x04 | 0x10
    return O.FLAG_SWITCH, 0x3C


def compare_faces(u, bc, op, gvm, gvp, gfl, tol_rel, max_tie_frac, geta=None, eta_exact=False, label=""):
    """u: [m][n] (or [n]) float64 cell averages the GPU saw; gvm, gvp, gfl (and geta) the GPU
    outputs as numpy arrays.  tol_rel: value bar relative to max |u| (per field).  Returns the
    share of switch-tied faces."""
    u = np.asarray(u, dtype=np.float64)
    squeeze = u.ndim == 1
    uu = u[None] if squeeze else u
    gvm, gvp, gfl = (np.asarray(x).reshape(uu.shape[0], -1) for x in (gvm, gvp, gfl))
    vm, vp, fl, eta, zr, _ = O.reconstruct(uu, bc, op, with_reason=True)
    sw, eno = masks(op.k)
    tie = ((fl & O.FLAG_SWITCH_TIE) != 0) | ((gfl & GPU_NEAR_TIE) != 0)
    frac = float(tie.mean())
    print(f"{label}: switch near ties on {frac:.4%} of {tie.size} faces")
    assert frac <= max_tie_frac, (label, frac)
    assert np.array_equal(gfl & eno, fl & eno), label
    assert np.array_equal((gfl & sw)[~tie], (fl & sw)[~tie]), label
    # replay the GPU's decisions: every face compares
    rvm, rvp, rfl, reta, rzr, _ = O.reconstruct(uu, bc, op, replay=gfl, with_reason=True)
    assert np.array_equal(rfl & (sw | eno), gfl & (sw | eno)), label
    for k in range(uu.shape[0]):
        scale = max(np.abs(uu[k]).max(), 1e-300)
        assert np.abs(gvm[k] - rvm[k]).max() <= tol_rel * scale, (label, k)
        assert np.abs(gvp[k] - rvp[k]).max() <= tol_rel * scale, (label, k)
    g_guard = (gfl & GPU_ZERO_GUARD) != 0
    g_bound = (gfl & GPU_ZERO_BOUND) != 0
    o_guard = (rzr & (O.ZERO_GUARD_L | O.ZERO_GUARD_R)) != 0
    o_bound = (rzr & (O.ZERO_BOUND_L | O.ZERO_BOUND_R)) != 0
    assert np.array_equal(g_guard, o_guard), label
    assert np.array_equal(g_bound, o_bound), label
    if geta is not None:
        geta = np.asarray(geta, dtype=np.float64).reshape(uu.shape[0], -1)
        if eta_exact:
            assert np.array_equal(geta, reta), label
        else:
            # a float shape parameter is the FP64 value rounded once: within one float ulp of it
            ulp = np.spacing(np.abs(reta).astype(np.float32)).astype(np.float64)
            assert np.all(np.abs(geta - reta) <= ulp), label
    return frac
