"""GPU association replay for the parity tests (Sec. 4.3 dense matching; the survey's protocol).

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
