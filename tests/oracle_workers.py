"""Oracle work for a pool of host processes (started with `spawn`): the FP64 blend of a chunk of
pixels compared with the GPU's results for them.  Imports numpy and the oracle only."""
from __future__ import annotations

import numpy as np

from oracle import oracle as O

_SHARED = {}


def init_blend(cam, proj, opacity, ids, ranges, idx, w, knife_edge):
    _SHARED.update(cam=cam, proj=proj, opacity=opacity, ids=ids, ranges=ranges, idx=idx, w=w, knife=knife_edge)


def blend_check(task):
    """task = (px, py, W [levels, n, L] f32, final_T [n], n_last [n]) from the GPU.  Returns the
    counts and worst ratios of the comparison: W within 1e-5 |W| + 1e-9 and final T within
    1e-5 |T| + 1e-9 on pixels whose decisions are not within 1e-4 of a threshold, the last
    contributor equal there; on the knife-edge pixels the largest W error."""
    px, py, Wg, Tg, ng = task
    s = _SHARED
    bl = O.blend(s["cam"], s["proj"], s["opacity"], s["ids"], s["ranges"], idx=s["idx"], w=s["w"], px=px, py=py,
                 C_out=Wg.shape[2])
    ok = bl.margin > s["knife"]
    Wg = Wg.astype(np.float64)
    err = np.abs(Wg[:, ok] - bl.out[:, ok])
    bound = 1e-5 * np.abs(bl.out[:, ok]) + 1e-9
    terr = np.abs(Tg[ok].astype(np.float64) - bl.final_T[ok])
    tbound = 1e-5 * np.abs(bl.final_T[ok]) + 1e-9
    knife = ~ok
    return {"pixels": int(px.size), "checked": int(ok.sum()),
            "w_worst": float((err / bound).max()) if err.size else 0.0,
            "w_bad": int((err > bound).sum()),
            "t_worst": float((terr / tbound).max()) if terr.size else 0.0,
            "n_last_mismatch": int((ng[ok].astype(np.int64) != bl.n_last[ok]).sum()),
            "knife": int(knife.sum()),
            "knife_err": float(np.abs(Wg[:, knife] - bl.out[:, knife]).max()) if knife.any() else 0.0,
            "contributions": int(bl.n_contrib.sum())}
