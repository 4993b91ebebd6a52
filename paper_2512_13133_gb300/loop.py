"""Coarse-to-fine clustering with a low-resolution coarse stage (Sec. 3.1
stages 2-4): the relaxed graph comes from the clips rasterised at a coarser
pitch (fewer pixels, so cheaper gates and alignment) with relaxed thresholds,
and each member is accepted only by the strict full-resolution decision
against its representative.  Every step is a C-ABI call of libpcl; this
module only sequences them.

The coarse stage is lossy on purpose (a pair that passes at full resolution
but is screened out at the coarse one never enters the graph); what it
keeps is the loop's guarantee: every member passes the strict test against
its representative.
"""
from __future__ import annotations

import numpy as np

from . import (MODE_COSINE, MODE_EDGE, F_ALIGNED, F_EDGE_VERIFY_FAIL, alloc_clipset, candidates, match,
               params, pcl_cluster_loop, pcl_rasterize, records_to_numpy)


def coarse_params(P, factor: int = 2, delta_cos: int = 2, delta_edge: int = 2):
    """parameters of the coarse stage: pitch x factor (same window and
    marker, so N and S shrink by the factor), cosine threshold num - delta
    over the same den, edge tolerance + delta dbu"""
    return params(P.window_dbu, P.pitch_dbu * factor, P.marker_dbu, P.cos_num - delta_cos, P.cos_den,
                  P.edge_tol_dbu + delta_edge, P.cos_engine, P.shift_rule, P.near_band, P.flags)


def coarse_to_fine(ctx, P, cs, rect_off, rects, mode: int = MODE_COSINE, factor: int = 2, delta_cos: int = 2,
                   delta_edge: int = 2):
    """Clusters of the clip set cs (rasterised under P; rect_off/rects its
    rectangles) with a coarse stage at pitch x factor.  Returns (rep_of,
    n_clusters, rounds, info) with info the pair counts of both stages."""
    Pc = coarse_params(P, factor, delta_cos, delta_edge)
    csc = alloc_clipset(Pc, rect_off, rects, with_spec=mode == MODE_COSINE)
    pcl_rasterize(ctx, Pc, csc)
    pairs, _ = candidates(ctx, Pc, mode, csc)
    rc = records_to_numpy(match(ctx, Pc, mode, csc, csc, pairs))
    rf = records_to_numpy(match(ctx, P, mode, cs, cs, pairs))
    if mode == MODE_EDGE:
        def ok(r, tol):
            good = ((r["flags"] & F_ALIGNED) > 0) & ((r["flags"] & F_EDGE_VERIFY_FAIL) == 0)
            return good & (r["score"].astype(np.int64) <= tol)
        relaxed, strict = ok(rc, Pc.edge_tol_dbu), ok(rf, P.edge_tol_dbu)
    else:
        relaxed, strict = rc["pass_"] > 0, rf["pass_"] > 0
    pr = np.stack([rc["a"], rc["b"]], 1).astype(np.int64)
    rep, ncl, rounds = pcl_cluster_loop(pr, strict, relaxed, cs.n)
    return rep, ncl, rounds, {"coarse_pairs": int(len(pr)), "relaxed": int(relaxed.sum()), "strict": int(strict.sum())}
