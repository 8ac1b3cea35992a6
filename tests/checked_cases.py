"""Parity cases run against the checked build of the library (device bounds
checks compiled in): every sweep kernel, the repair, replica exchange and a
batch, each compared with the CPU oracle, then the library's record of failed
checks, which must be empty.  Run by tests/test_gpu_device_checks.py in a
fresh interpreter with QPATH_LIBRARY pointing at libqpath_checked.so; prints
one JSON line and exits non-zero on any mismatch."""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import torch  # noqa: E402

import oracle  # noqa: E402
from oracle import pt_ref, repair_ref  # noqa: E402
from paper_2608_25376_gb300 import inputs, qpath  # noqa: E402

K = qpath


def anneal(h, R, S, seed, kernel):
    n = h.info["n"]
    st = torch.zeros((R, n), dtype=torch.uint8, device="cuda")
    E = torch.zeros(R, dtype=torch.int64, device="cuda")
    B = torch.zeros(R, dtype=torch.int64, device="cuda")
    qpath.qp_anneal_ex(h, R, qpath.schedule(S), seed, None, st, E, B, kernel=kernel,
                       stream=torch.cuda.current_stream())
    torch.cuda.synchronize()
    return st.cpu().numpy(), E.cpu().numpy(), B.cpu().numpy()


def same(got, ref):
    st, E, B = got
    return bool((st == ref.states).all() and (E == ref.energies).all() and (B == ref.best).all())


def main():
    assert os.environ.get("QPATH_LIBRARY"), "run with QPATH_LIBRARY set to the checked build"
    enabled, w = qpath.qp_device_checks()
    assert enabled, "the loaded library was built without device checks"
    oracle.build()
    results = {}
    structured = [("rows", K.QP_KERNEL_STRUCTURED_ROWS, 512), ("flat", K.QP_KERNEL_STRUCTURED_FLAT, 4096),
                  ("group", K.QP_KERNEL_STRUCTURED_GROUP, 128)]
    fields = [("3x3", inputs.rect(3, 3), {}), ("6x6-p0.2", inputs.obstacles(6, 6, 0.2, seed=3, start=14), {}),
              ("10x10-p0.1", inputs.obstacles(10, 10, 0.1, seed=1), {}),
              ("5x5-int32", inputs.obstacles(5, 5, 0.1, seed=4), {"scale": 10000}),
              ("18x18-p0.1", inputs.obstacles(18, 18, 0.1, seed=8, start=5), {}),
              ("16x32", inputs.rect(16, 32), {}), ("24x24-p0.05", inputs.obstacles(24, 24, 0.05, seed=8), {})]
    for name, f, kw in fields:
        P = oracle.Problem(f.rows, f.cols, f.free_mask, f.start, **kw)
        R, S = (16, 60) if P.C <= 128 else (3, 4)
        ref = oracle.anneal_structured(P, R, S, seed=3)
        dense = P.C <= 36
        h = qpath.qp_build_qubo(f, flags=K.QP_STRUCTURED | (K.QP_DENSE if dense else 0), **kw)
        for kname, kernel, cmax in structured:
            if P.C <= cmax:
                results[f"{name}/{kname}"] = same(anneal(h, R, S, 3, kernel), ref)
        if dense:
            results[f"{name}/dense"] = same(anneal(h, R, S, 3, K.QP_KERNEL_DENSE), ref)
    # repair of annealed states
    f = inputs.obstacles(6, 6, 0.15, seed=2)
    P = oracle.Problem(f.rows, f.cols, f.free_mask, f.start)
    h = qpath.qp_build_qubo(f)
    R = 32
    ref = oracle.anneal_structured(P, R, 30, seed=3)
    paths, lens, stat = np.zeros((R, P.C), np.int32), np.zeros(R, np.int64), np.zeros(R, np.int32)
    qpath.qp_repair_batch(h, R, ref.states, -1, paths, lens, stat)
    dl = P.d.tolist()
    ok = True
    for r in range(R):
        p_ref, l_ref, s_ref = repair_ref.repair(ref.states[r].tolist(), dl, P.C, P.start_cell, -1)
        ok &= paths[r].tolist() == p_ref and int(lens[r]) == l_ref and int(stat[r]) == s_ref
    results["repair"] = bool(ok)
    # replica exchange
    G, M = 2, 4
    out = pt_ref.anneal_pt(P, G, M, 10.0, 1000.0, 5, 4, seed=3)
    pst, pE = np.zeros((G * M, P.n), np.uint8), np.zeros(G * M, np.int64)
    qpath.qp_anneal_pt(h, G, qpath.pt_schedule(M, 10.0, 1000.0, 5, 4), 3, None, pst, pE)
    results["replica_exchange"] = bool((pE == out["energies"]).all() and (pst == out["states"]).all())
    # a batch of uneven fields
    fs = [inputs.obstacles(4, 7, 0.1, seed=11), inputs.obstacles(9, 6, 0.2, seed=12), inputs.rect(5, 5)]
    hs = [qpath.qp_build_qubo(ff) for ff in fs]
    Rb, Sb = 8, 30
    sts = [torch.zeros((Rb, hh.info["n"]), dtype=torch.uint8, device="cuda") for hh in hs]
    Es = [torch.zeros(Rb, dtype=torch.int64, device="cuda") for _ in hs]
    qpath.qp_anneal_batch(hs, Rb, qpath.schedule(Sb), 5, sts, Es, stream=torch.cuda.current_stream())
    torch.cuda.synchronize()
    ok = True
    for i, ff in enumerate(fs):
        Pf = oracle.Problem(ff.rows, ff.cols, ff.free_mask, ff.start)
        rf = oracle.anneal_structured(Pf, Rb, Sb, seed=5 + i)
        ok &= bool((sts[i].cpu().numpy() == rf.states).all() and (Es[i].cpu().numpy() == rf.energies).all())
    results["batch"] = ok
    enabled, first_failure = qpath.qp_device_checks()
    print(json.dumps({"enabled": enabled, "first_failure": first_failure, "results": results}))
    return 0 if enabled and first_failure == 0 and all(results.values()) else 1


if __name__ == "__main__":
    sys.exit(main())
