"""Accuracy of scene-flow results against ground truth, in the form of the
KITTI scene-flow benchmark's figures that Sec. 4 reports (Table 1):

- D1: disparity at t (the reference view) -> error |d0 - d0*|;
- D2: disparity at t+1 of the same 3D point, at the reference pixel ->
  error |d1 - d1*|;
- Fl: the 2D flow -> error ||(u, v) - (u*, v*)||;
- SF: a pixel is a scene-flow outlier if it is an outlier in any of the
  three.

A value is an outlier when its error exceeds both 3 px and 5 % of the true
magnitude (the benchmark's rule).  The rates here are over the pixels the
method keeps (its validity mask), with the density (kept pixels over all
pixels) beside them: the paper's method is sparse by design (Sec. 3.3).  The synthetic scenes supply the ground truth
(``synth.Quad.gt_disp0``, ``gt_disp1``, ``gt_flow``).

Sec. 4 also reports a dense variant ("All" in Table 1), which the benchmark
makes from a sparse submission by filling the gaps of each map with
background values.  ``fill_background`` is this package's reading of that
step: within each row, a run of missing values between two kept ones takes
the smaller of the two (the farther surface for a disparity), a run at a
row end takes its one neighbour; rows with nothing kept then take values
the same way along their column.  ``scene_flow_accuracy_dense`` fills d0 and
d1 so, takes (u, v) from the input flow, and scores every pixel.

Host-side evaluation on tensors (any device); no part of the hot path."""
from __future__ import annotations

import torch

ABS_PX = 3.0
REL = 0.05


def outliers(err: torch.Tensor, true_mag: torch.Tensor, abs_px: float = ABS_PX, rel: float = REL):
    """Boolean mask: error above abs_px and above rel times the true magnitude."""
    return (err > abs_px) & (err > rel * true_mag.abs())


def scene_flow_accuracy(s4, valid, gt_disp0, gt_disp1, gt_flow, abs_px: float = ABS_PX, rel: float = REL):
    """s4: [H][W][4] (u, v, d0, d1); valid: [H][W] (nonzero = kept);
    gt_disp0, gt_disp1: [H][W]; gt_flow: [H][W][2].  Pixels whose ground
    truth is not finite count as neither kept nor evaluated.  Returns
    {"density", "D1", "D2", "Fl", "SF"} (rates over the kept pixels)."""
    s4 = torch.as_tensor(s4, dtype=torch.float64)
    dev = s4.device
    gt0 = torch.as_tensor(gt_disp0, dtype=torch.float64, device=dev)
    gt1 = torch.as_tensor(gt_disp1, dtype=torch.float64, device=dev)
    gtf = torch.as_tensor(gt_flow, dtype=torch.float64, device=dev)
    has_gt = torch.isfinite(gt0) & torch.isfinite(gt1) & torch.isfinite(gtf).all(dim=-1)
    kept = torch.as_tensor(valid, device=dev).to(torch.bool) & has_gt
    n_kept = int(kept.sum())
    o1 = outliers((s4[..., 2] - gt0).abs(), gt0, abs_px, rel)
    o2 = outliers((s4[..., 3] - gt1).abs(), gt1, abs_px, rel)
    ofl = outliers(torch.linalg.vector_norm(s4[..., :2] - gtf, dim=-1), torch.linalg.vector_norm(gtf, dim=-1),
                   abs_px, rel)
    osf = o1 | o2 | ofl

    def rate(o):
        return float(o[kept].sum()) / n_kept if n_kept else 0.0

    return {"density": n_kept / max(int(has_gt.sum()), 1), "D1": rate(o1), "D2": rate(o2), "Fl": rate(ofl),
            "SF": rate(osf)}


def _fill_rows(a: torch.Tensor) -> torch.Tensor:
    """Row-wise background fill of the NaN entries of a 2-D tensor."""
    H, W = a.shape
    ok = ~torch.isnan(a)
    idx = torch.arange(W, device=a.device).expand(H, W)
    # index of the nearest kept entry at or left of / at or right of each position
    left = torch.where(ok, idx, torch.full_like(idx, -1)).cummax(dim=1).values
    right_f = torch.where(ok, W - 1 - idx, torch.full_like(idx, -1)).flip(1).cummax(dim=1).values.flip(1)
    right = torch.where(right_f >= 0, W - 1 - right_f, torch.full_like(idx, -1))
    lv = torch.gather(a, 1, left.clamp(min=0))
    rv = torch.gather(a, 1, right.clamp(min=0))
    has_l, has_r = left >= 0, right >= 0
    both = torch.minimum(lv, rv)
    filled = torch.where(has_l & has_r, both, torch.where(has_l, lv, torch.where(has_r, rv, a)))
    return torch.where(ok, a, filled)


def fill_background(a) -> torch.Tensor:
    """Background fill of a 2-D map whose missing values are NaN: along the
    rows first, then along the columns for whatever is still missing."""
    a = torch.as_tensor(a, dtype=torch.float64)
    rows = _fill_rows(a)
    cols = _fill_rows(rows.t().contiguous()).t()
    return torch.where(torch.isnan(rows), cols, rows)


def scene_flow_accuracy_dense(s4, flow, gt_disp0, gt_disp1, gt_flow, abs_px: float = ABS_PX, rel: float = REL):
    """The figures of scene_flow_accuracy for a densified result: d0 and d1
    of s4 filled by fill_background, (u, v) from the input flow everywhere.
    Density is then 1 wherever any value was kept in the frame."""
    s4 = torch.as_tensor(s4, dtype=torch.float64)
    dev = s4.device
    d0 = fill_background(s4[..., 2])
    d1 = fill_background(s4[..., 3])
    uv = torch.as_tensor(flow, dtype=torch.float64, device=dev)
    dense = torch.cat([uv, d0.unsqueeze(-1), d1.unsqueeze(-1)], dim=-1)
    kept = (~torch.isnan(d0) & ~torch.isnan(d1)).to(torch.uint8)
    return scene_flow_accuracy(dense, kept, gt_disp0, gt_disp1, gt_flow, abs_px, rel)
