"""Shared test helpers: unpacking bit columns, oracle dispatch."""
import numpy as np

from oracle import statevector as osv
from oracle import symft as osymft
from oracle import tableau as otab
from oracle.circuit import parse as oparse


def unpack(cols, shots):
    """(ncol, W) uint64 packed columns -> (shots, ncol) uint8 bits."""
    cols = np.ascontiguousarray(np.asarray(cols, dtype=np.uint64))
    ncol = cols.shape[0]
    if ncol == 0:
        return np.zeros((shots, 0), dtype=np.uint8)
    b = np.unpackbits(cols.view(np.uint8).reshape(ncol, -1), axis=1, bitorder="little")
    return b[:, :shots].T.copy()


def padding_is_zero(cols, shots):
    cols = np.asarray(cols, dtype=np.uint64)
    if cols.size == 0 or shots % 64 == 0:
        return True
    tail = cols[:, -1] >> np.uint64(shots % 64)
    return bool((tail == 0).all())


def oracle_sample(text, seed, shots, postselect=0, kind="auto", post_dets=None):
    c = oparse(text)
    has_rot = any(op.kind == "rot" for op in c.ops)
    if kind == "auto":
        kind = "symft" if has_rot else "tableau"
    if kind == "tableau":
        return otab.sample(c, seed, shots, postselect, post_dets=post_dets)
    if kind == "sv":
        return osv.sample(c, seed, shots, postselect, post_dets=post_dets)
    return osymft.sample(c, seed, shots, postselect, post_dets=post_dets)


def gpu_sample(text, shots, seed, shot_offset=0, precision=0, postselect=0, host=False,
               post_dets=None):
    import torch
    import paper_2607_28600_b300 as S
    plan = S.symft_compile(text, postselect=postselect, post_dets=post_dets)
    info = plan.info
    W = (shots + 63) // 64
    if host:
        meas = np.zeros((info["n_records"], W), dtype=np.uint64)
        det = np.zeros((info["n_dets"], W), dtype=np.uint64)
        obs = np.zeros((info["n_obs"], W), dtype=np.uint64)
        disc = np.zeros((W,), dtype=np.uint64)
        S.symft_sample_ex(plan, shots, seed, shot_offset=shot_offset,
                          meas_out=meas if meas.size else None, det_out=det if det.size else None,
                          obs_out=obs if obs.size else None, discard_out=disc,
                          precision=precision, out_location=S.OUT_HOST, check=True)
        return plan, meas, det, obs, disc
    meas, det, obs, disc = S.sample_to_tensors(plan, shots, seed, shot_offset=shot_offset,
                                               precision=precision)
    torch.cuda.synchronize()
    return (plan, meas.cpu().numpy().view(np.uint64), det.cpu().numpy().view(np.uint64),
            obs.cpu().numpy().view(np.uint64), disc.cpu().numpy().view(np.uint64))
