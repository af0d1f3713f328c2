"""Shared test helper: which block levels sit safely away from the VLM thresholds."""

import numpy as np


def robust_level_mask(stats, level_map, lambda_batch, block, max_mip, te, tc, cm, eps=1e-4):
    """True where the oracle's block level is not within eps of any deciding threshold."""
    n_batch, nbz, nbx = level_map.shape
    rp, rf = [], []
    for st in stats:
        L = st["iod_eta"].shape[0]
        with np.errstate(invalid="ignore"):
            p = ((st["iod_eta"] < te * (1 - eps)) & (st["iod_chi"] < tc * (1 - eps))) | (st["chi_ds"] < cm * (1 - eps))
            f = ((st["iod_eta"] > te * (1 + eps)) | (st["iod_chi"] > tc * (1 + eps))) & \
                ((st["chi_ds"] > cm * (1 + eps)) if cm > 0 else True)   # cm <= 0: no always-average rule
        side = p.shape[1] // nbz

        def per_batch(a, red):
            blk = red(a.reshape(L, nbz, side, nbx, side), axis=(2, 4))
            return np.stack([red(blk[b * lambda_batch:(b + 1) * lambda_batch], axis=0) for b in range(n_batch)])
        rp.append(per_batch(p, np.all))
        rf.append(per_batch(f, np.any))
    ok = np.ones(level_map.shape, dtype=bool)
    for b in range(n_batch):
        for bz in range(nbz):
            for bx in range(nbx):
                L_ = level_map[b, bz, bx]
                if L_ < 0:
                    continue
                good = all(rp[m - 1][b, bz, bx] for m in range(1, L_ + 1))
                if L_ < max_mip:
                    good = good and rf[L_][b, bz, bx]
                ok[b, bz, bx] = good
    return ok


def robust_level_mask3(stats, level_map, lambda_batch, max_mip, te, tc, cm, eps=1e-4):
    """3D form of :func:`robust_level_mask`: level_map ``[n_batch][nbz][nby][nbx]``."""
    n_batch, nbz, nby, nbx = level_map.shape
    rp, rf = [], []
    for st in stats:
        L = st["iod_eta"].shape[0]
        with np.errstate(invalid="ignore"):
            p = ((st["iod_eta"] < te * (1 - eps)) & (st["iod_chi"] < tc * (1 - eps))) | (st["chi_ds"] < cm * (1 - eps))
            f = ((st["iod_eta"] > te * (1 + eps)) | (st["iod_chi"] > tc * (1 + eps))) & \
                ((st["chi_ds"] > cm * (1 + eps)) if cm > 0 else True)   # cm <= 0: no always-average rule
        s = p.shape[1] // nbz

        def per_batch(a, red):
            blk = red(a.reshape(L, nbz, s, nby, s, nbx, s), axis=(2, 4, 6))
            return np.stack([red(blk[b * lambda_batch:(b + 1) * lambda_batch], axis=0) for b in range(n_batch)])
        rp.append(per_batch(p, np.all))
        rf.append(per_batch(f, np.any))
    ok = np.ones(level_map.shape, dtype=bool)
    for idx in np.ndindex(*level_map.shape):
        L_ = level_map[idx]
        if L_ < 0:
            continue
        good = all(rp[m - 1][idx] for m in range(1, L_ + 1))
        if L_ < max_mip:
            good = good and rf[L_][idx]
        ok[idx] = good
    return ok


def candidate_levels(stats, level_map, lambda_batch, block, max_mip, te, tc, cm, eps=1e-4):
    """Every level a block-batch may take when its decisions near a threshold go
    either way: {index: [levels]} for the block-batches that are not robust.

    Level l is a candidate when no decision of levels 1..l fails robustly (each
    level's groups can all pass) and, below max_mip, level l + 1 does not pass
    robustly (it can fail)."""
    n_batch, nbz, nbx = level_map.shape
    rp, rf = [], []
    for st in stats:
        L = st["iod_eta"].shape[0]
        with np.errstate(invalid="ignore"):
            p = ((st["iod_eta"] < te * (1 - eps)) & (st["iod_chi"] < tc * (1 - eps))) | (st["chi_ds"] < cm * (1 - eps))
            f = ((st["iod_eta"] > te * (1 + eps)) | (st["iod_chi"] > tc * (1 + eps))) & \
                ((st["chi_ds"] > cm * (1 + eps)) if cm > 0 else True)   # cm <= 0: no always-average rule
        side = p.shape[1] // nbz

        def per_batch(a, red):
            blk = red(a.reshape(L, nbz, side, nbx, side), axis=(2, 4))
            return np.stack([red(blk[b * lambda_batch:(b + 1) * lambda_batch], axis=0) for b in range(n_batch)])
        rp.append(per_batch(p, np.all))
        rf.append(per_batch(f, np.any))
    robust = robust_level_mask(stats, level_map, lambda_batch, block, max_mip, te, tc, cm, eps)
    out = {}
    for idx in zip(*np.nonzero(~robust)):
        cands = []
        for lv in range(max_mip + 1):
            can_pass = all(not rf[m - 1][idx] for m in range(1, lv + 1))
            can_stop = lv == max_mip or not rp[lv][idx]
            if can_pass and can_stop:
                cands.append(lv)
        out[tuple(int(v) for v in idx)] = cands
    return out


def robust_level_mask_multi(stats_list, level_map, lambda_batch, block, max_mip, te, tc, cm, eps=1e-4):
    """:func:`robust_level_mask` for a level test made of several evaluations that
    must all pass (the moving-medium builds with directional tests): a group passes
    robustly when every evaluation passes robustly, and fails robustly when some
    evaluation fails robustly.  ``stats_list``: one per-level stats list per evaluation."""
    n_batch, nbz, nbx = level_map.shape
    rp, rf = None, None
    for stats in stats_list:
        rpe, rfe = [], []
        for st in stats:
            L = st["iod_eta"].shape[0]
            with np.errstate(invalid="ignore"):
                p = ((st["iod_eta"] < te * (1 - eps)) & (st["iod_chi"] < tc * (1 - eps))) | (st["chi_ds"] < cm * (1 - eps))
                f = ((st["iod_eta"] > te * (1 + eps)) | (st["iod_chi"] > tc * (1 + eps))) & \
                    ((st["chi_ds"] > cm * (1 + eps)) if cm > 0 else True)
            side = p.shape[1] // nbz

            def per_batch(a, red):
                blk = red(a.reshape(L, nbz, side, nbx, side), axis=(2, 4))
                return np.stack([red(blk[b * lambda_batch:(b + 1) * lambda_batch], axis=0) for b in range(n_batch)])
            rpe.append(per_batch(p, np.all))
            rfe.append(per_batch(f, np.any))
        rp = rpe if rp is None else [a & b for a, b in zip(rp, rpe)]
        rf = rfe if rf is None else [a | b for a, b in zip(rf, rfe)]
    ok = np.ones(level_map.shape, dtype=bool)
    for idx in np.ndindex(*level_map.shape):
        L_ = level_map[idx]
        if L_ < 0:
            continue
        good = all(rp[m - 1][idx] for m in range(1, L_ + 1))
        if L_ < max_mip:
            good = good and rf[L_][idx]
        ok[idx] = good
    return ok
