"""GPU association replay for the parity tests (Sec. 4.3 dense matching).

The library takes its association decisions in FP32 and the oracle in FP64, so a few decisions
per million (those within FP32 rounding of a threshold: a projection next to a pixel boundary, a
distance or a normal cosine next to its gate) can go either way; both outcomes are correct there.
To compare the residual, Jacobian and normal-equation arithmetic element by element, the oracle
replays the library's decisions, fetched through bf_debug_association at the oracle's own poses,
after checking them: every decision must equal the oracle's except on ties
(oracle.association.CheckedReplay raises otherwise), and the number of flips is reported.
"""
from oracle import association


# 16-bit frame storage: a stored normal component may sit one 16-bit ulp away from the oracle's
# (a value whose FP32 and FP64 results straddle a rounding boundary), which moves the normal cosine
# by up to about two ulps of 1
EPS_N_STORAGE = {None: association.EPS_N, "fp32": association.EPS_N, "bf16": 2.0 ** -6, "fp16": 2.0 ** -9}


def from_ctx(ctx, frame_ids, W, H, storage=None, **params):
    """CheckedReplay whose decisions come from the library context ``ctx``; local frame index k of
    the oracle's solve is the context's frame frame_ids[k]."""
    ids = [int(f) for f in frame_ids]

    def fetch(i, j, poses):
        return ctx.association(ids[i], ids[j], poses[i], poses[j], **params)

    eps = (association.EPS_PX, association.EPS_D, EPS_N_STORAGE[storage])
    return association.CheckedReplay(fetch, W, H, eps)


class Recorded(association.CheckedReplay):
    """The decisions the library took in its last recorded solve on ``ctx`` (bf_debug_record_association),
    per dense evaluation: the oracle checks each against its own FP64 association at the poses the
    library evaluated at, then replays it in its own Gauss-Newton loop (at its own poses), so that
    every iteration of both solves sums the same pixels."""

    def __init__(self, ctx, frame_ids, W, H, storage=None):
        super().__init__(self._fetch, W, H, (association.EPS_PX, association.EPS_D, EPS_N_STORAGE[storage]))
        self.ctx, self.ids = ctx, [int(f) for f in frame_ids]
        self._key, self._val = None, None

    def _get(self, i, j):
        key = (self.iteration, i, j)
        if key != self._key:
            self._key, self._val = key, self.ctx.recorded_association(self.iteration, self.ids[i], self.ids[j])
        return self._val

    def _fetch(self, i, j, poses):
        return self._get(i, j)[0]

    def check_poses(self, i, j):
        _, Pi, Pj = self._get(i, j)
        return Pi, Pj


def recorded_solve(ctx, frame_ids, solve, oracle_frames, intr, init, sparse_pairs, params, storage=None, pmap=None,
                   frame_keys=None):
    """Run ``solve()`` (one single-problem solve on ctx) with the association recorded, then the
    oracle's Gauss-Newton solve from ``init`` on the recorded decisions.  Returns (the library's
    stats, its poses of frame_ids, the oracle's result with ``.replay`` = the Recorded provider)."""
    from oracle import solver
    ctx.record_association(True)
    try:
        st = solve()
        poses = ctx.get_poses(frame_ids)
        rep = Recorded(ctx, frame_ids, intr["W"], intr["H"], storage)
        ref = solver.gauss_newton(oracle_frames, intr, init, sparse_pairs, params, assoc=rep, pmap=pmap,
                                  frame_keys=frame_keys)
    finally:
        ctx.record_association(False)
    ref.replay = rep
    return st, poses, ref
