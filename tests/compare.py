"""Element-wise comparison of library results with the oracle's (both in the
oracle's layout: per-cell arrays in input order plus a CSR of faces)."""
import numpy as np


def compare(got, ref, rtol, cells=None):
    """Returns a dict of mismatch counts and max relative errors.  Topology
    (status, V/E/F counts, neighbour ids and images, face orders) must be
    identical.  Volume, area and centroid errors are relative to the cell's
    own scale: max(|V|, 1e-4 R^d) for the volume, max(|A|, 1e-3 R^(d-1)) for
    the area and that volume scale^(1/d) for the centroid (R: the cell's
    largest vertex distance).  For ordinary cells this is plain relative
    error; a sliver cell far thinner than R (possible in radical
    tessellations) is measured against R, since no floating-point form can
    hold its tiny volume to a relative bound."""
    n = len(ref["vol"])
    idx = np.arange(n) if cells is None else np.asarray(cells)
    rep = {}
    st_g = got["status"][idx].astype(np.int64)
    st_r = ref["status"].astype(np.int64)
    rep["status_mismatch"] = int((st_g != st_r).sum())
    ok = st_r == 0
    for k in ("nv", "ne", "nf"):
        rep[k + "_mismatch"] = int((got[k][idx][ok] != ref[k][ok]).sum())
    d = ref["centroid"].shape[1]
    # faces per cell, compared for all cells at once: cells whose face counts
    # agree are compared face by face through index arrays
    fo_r = np.asarray(ref["face_off"], dtype=np.int64)
    fo_g = np.asarray(got["face_off"], dtype=np.int64)
    cnt_r = np.diff(fo_r)
    cnt_g = (fo_g[1:] - fo_g[:-1])[idx]
    same = ok & (cnt_r == cnt_g)
    bad_faces = int((ok & (cnt_r != cnt_g)).sum())
    sel = np.nonzero(same)[0]
    c = cnt_r[sel]
    tot = int(c.sum())
    if tot:
        cell = np.repeat(np.arange(len(sel)), c)
        within = np.arange(tot) - np.repeat(np.cumsum(c) - c, c)
        fr = fo_r[sel][cell] + within
        fg = fo_g[idx[sel]][cell] + within
        img_r = np.asarray(ref["nbr_img"])[:, :d]
        img_g = np.asarray(got["nbr_img"])[:, :d]
        diff = ((np.asarray(ref["nbr_id"])[fr] != np.asarray(got["nbr_id"])[fg]) |
                np.any(img_r[fr] != img_g[fg], axis=1) |
                (np.asarray(ref["face_order"])[fr] != np.asarray(got["face_order"])[fg]))
        bad_faces += int(len(np.unique(cell[diff])))
    rep["face_mismatch"] = bad_faces
    vr = ref["vol"][ok]
    vg = got["vol"][idx][ok]
    R = ref["rmax"][ok]
    vscale = np.maximum(np.abs(vr), 1e-4 * R ** d)
    rel = np.abs(vg - vr) / np.maximum(vscale, 1e-300)
    rep["vol_max_rel"] = float(rel.max()) if rel.size else 0.0
    rep["vol_rms_rel"] = float(np.sqrt(np.mean(rel ** 2))) if rel.size else 0.0
    ar = ref["area"][ok]
    ascale = np.maximum(np.abs(ar), 1e-3 * R ** (d - 1))
    arel = np.abs(got["area"][idx][ok] - ar) / np.maximum(ascale, 1e-300)
    rep["area_max_rel"] = float(arel.max()) if arel.size else 0.0
    rep["area_rms_rel"] = float(np.sqrt(np.mean(arel ** 2))) if arel.size else 0.0
    size = np.maximum(vscale, 1e-300) ** (1.0 / d)
    cd = np.linalg.norm(got["centroid"][idx][ok] - ref["centroid"][ok], axis=1) / size
    rep["centroid_max_rel"] = float(cd.max()) if cd.size else 0.0
    rep["centroid_rms_rel"] = float(np.sqrt(np.mean(cd ** 2))) if cd.size else 0.0
    rep["topology_ok"] = (rep["status_mismatch"] == 0 and rep["nv_mismatch"] == 0 and
                          rep["ne_mismatch"] == 0 and rep["nf_mismatch"] == 0 and bad_faces == 0)
    rep["values_ok"] = (rep["vol_max_rel"] <= rtol and rep["area_max_rel"] <= rtol and
                        rep["centroid_max_rel"] <= rtol)
    return rep
