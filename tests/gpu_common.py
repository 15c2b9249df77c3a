"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def run_fmm(w, p=None, theta=None, ncrit=None, m2l_mode=0, ksig=5.0, sigma_arr=None, images=None, outputs=None,
            sigma_rule=None, p2p_pair_max=None, split_tie=None, p2p_tpl=None, stretching=True):
    import torch
    from paper_1106_5273_gb300 import Plan, Params
    pos, gam = w["pos"], w["gamma"]
    n = pos.shape[0]
    kw = dict(p=p or w.get("p", 6), theta=theta or w.get("theta", 0.5), ncrit=ncrit or w.get("ncrit", 32),
              sigma_sep=ksig, m2l_mode=m2l_mode)
    if w.get("periodic"):
        kw.update(periodic=1, box_min=w["box_min"], box_len=w["box_len"], images=images or w.get("images", 3))
    if outputs is not None:
        kw.update(outputs=outputs)
    if sigma_rule is not None:
        kw.update(sigma_rule=sigma_rule)
    if p2p_pair_max is not None:
        kw.update(p2p_pair_max=p2p_pair_max)
    if split_tie is not None:
        kw.update(split_tie=split_tie)
    if p2p_tpl is not None:
        kw.update(p2p_tpl=p2p_tpl)
    plan = Plan(max(n, 1), Params.default(**kw))
    dp, dg = to_dev(pos), to_dev(gam)
    ds = to_dev(sigma_arr) if sigma_arr is not None else None
    u, s = plan.eval(dp, dg, sigma=ds, sigma_uniform=float(w["sigma"]), stretching=stretching)
    torch.cuda.synchronize()
    s = s.cpu().numpy().astype(np.float64) if s is not None else None
    return plan, u.cpu().numpy().astype(np.float64), s


def per_target_error(a, ref, floor=0.1):
    """max_i |a_i - ref_i| / (|ref_i| + floor * rms(ref)): the error of the worst
    target relative to its own magnitude, floored at a fraction of the rms
    magnitude so that targets where the field nearly vanishes do not divide
    by zero."""
    a = np.asarray(a, np.float64)
    ref = np.asarray(ref, np.float64)
    rms = np.linalg.norm(ref) / np.sqrt(max(ref.shape[0], 1))
    return float((np.linalg.norm(a - ref, axis=1) / (np.linalg.norm(ref, axis=1) + floor * rms)).max())
