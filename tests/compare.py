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
    # faces per cell
    bad_faces = 0
    for j, i in enumerate(idx):
        if not ok[j]:
            continue
        a, b = ref["face_off"][j], ref["face_off"][j + 1]
        ga, gb = got["face_off"][i], got["face_off"][i + 1]
        if (b - a) != (gb - ga):
            bad_faces += 1
            continue
        if not (np.array_equal(ref["nbr_id"][a:b], got["nbr_id"][ga:gb])
                and np.array_equal(np.asarray(ref["nbr_img"][a:b])[:, :d],
                                   np.asarray(got["nbr_img"][ga:gb])[:, :d])
                and np.array_equal(ref["face_order"][a:b], got["face_order"][ga:gb])):
            bad_faces += 1
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
    size = np.maximum(vscale, 1e-300) ** (1.0 / d)
    cd = np.linalg.norm(got["centroid"][idx][ok] - ref["centroid"][ok], axis=1) / size
    rep["centroid_max_rel"] = float(cd.max()) if cd.size else 0.0
    rep["topology_ok"] = (rep["status_mismatch"] == 0 and rep["nv_mismatch"] == 0 and
                          rep["ne_mismatch"] == 0 and rep["nf_mismatch"] == 0 and bad_faces == 0)
    rep["values_ok"] = (rep["vol_max_rel"] <= rtol and rep["area_max_rel"] <= rtol and
                        rep["centroid_max_rel"] <= rtol)
    return rep
