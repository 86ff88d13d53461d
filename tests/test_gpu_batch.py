"""Batched small-problem Lanczos against the oracle, and the batch invariants:
a problem's result does not depend on the rest of the batch nor on the launch
chunk (bit for bit); each problem stops where the oracle's Lanczos stops."""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_util import ctx, pair
from paper_2307_13222_gb300 import hphi
from workloads import (chain, ladder, heisenberg_terms, hubbard_terms, random_vectors, configs, uniform_couplings)

pytestmark = pytest.mark.gpu


def _problems():
    cfg = configs.heisenberg_chain16()
    out = [("chain16", cfg["model"], 16, 8, 0, cfg["terms"], cfg["seed"]),
           ("chain10_rand", "SPIN_HALF", 10, 5, 0, heisenberg_terms(chain(10), uniform_couplings(10, 0.5, 1.5, 3)), 4),
           ("chain11_sz", "SPIN_HALF", 11, 4, 0, [("XXZ", i, (i + 1) % 11, 0, 0.7, 1.3) for i in range(11)], 5),
           ("ladder6", "SPIN_HALF", 12, 6, 0, heisenberg_terms(ladder(6), 1.0), 6),
           ("gc10", "SPIN_HALF_GC", 10, 0, 0, heisenberg_terms(chain(10), uniform_couplings(10, 0.5, 1.5, 8)), 7),
           ("hub6", "HUBBARD", 6, 3, 3, hubbard_terms(6, chain(6), t=1.0, U=4.0), 8),
           ("hub6V", "HUBBARD", 6, 3, 2, hubbard_terms(6, chain(6), t=1.0, U=6.0, V=0.7)
            + [("HOP", 0, 3, 0, 0.4, 0.0)], 9),
           # x (1.5 MB) stays in global memory, the rank tables go to shared memory
           ("chain20", "SPIN_HALF", 20, 10, 0, heisenberg_terms(chain(20), 1.0), 10),
           # rank tables (192 KB) stay in global memory, x goes to shared memory
           ("chain28_2up", "SPIN_HALF", 28, 2, 0, heisenberg_terms(chain(28), uniform_couplings(28, 0.5, 1.5, 2)), 11),
           ("hub10", "HUBBARD", 10, 5, 5, hubbard_terms(10, chain(10), t=1.0, U=8.0), 12)]
    return out


def _build(problems):
    ms, hs, vs = [], [], []
    for name, model, N, nu, nd, terms, seed in problems:
        m, b, h = pair(model, N, nu, nd, terms)
        ms.append(m)
        hs.append((b, h))
        vs.append(torch.from_numpy(random_vectors(m.dim, 1, seed)[:, 0]).cuda())
    return ms, hs, vs


def test_mixed_batch_against_oracle():
    probs = _problems()
    ms, hs, vs = _build(probs)
    gss = [torch.empty_like(v) for v in vs]
    res = hphi.hphi_lanczos_batch([h for _, h in hs], vs, 400, 1e-12, check_every=8, gs_outs=gss)
    for (name, *_), m, v, r, g in zip(probs, ms, vs, res, gss):
        ro = m.lanczos(v.cpu().numpy(), 400, 1e-12, want_gs=True)
        assert r["status"] == 0 and r["converged"], name
        assert abs(r["e0"] - ro["e0"]) <= 1e-10 * abs(ro["e0"]), (name, r["e0"], ro["e0"])
        assert abs(r["steps"] - ro["steps"]) <= 1, (name, r["steps"], ro["steps"])
        assert abs(np.dot(g.cpu().numpy(), ro["gs"])) >= 1 - 1e-10, name
        assert r["resid"] < 1e-9, name
        if m.dim <= 2000:
            w = np.linalg.eigvalsh(O.dense_matrix(m))
            assert abs(r["e0"] - w[0]) <= 1e-10 * abs(w[0]), name


def test_result_independent_of_batch_and_chunk():
    probs = _problems()
    ms, hs, vs = _build(probs)
    H = [h for _, h in hs]
    g_alone = torch.empty_like(vs[0])
    alone = hphi.hphi_lanczos_batch([H[0]], [vs[0]], 400, 1e-12, check_every=1, gs_outs=[g_alone])[0]
    for chunk in (3, 16):
        gss = [torch.empty_like(v) for v in vs]
        res = hphi.hphi_lanczos_batch(H, vs, 400, 1e-12, check_every=chunk, gs_outs=gss)
        assert res[0]["e0"] == alone["e0"] and res[0]["steps"] == alone["steps"]
        assert torch.equal(gss[0], g_alone)
    # the same Hamiltonian several times with different start vectors
    seeds = [11, 12, 13, 14]
    v2 = [torch.from_numpy(random_vectors(ms[0].dim, 1, s)[:, 0]).cuda() for s in seeds]
    res = hphi.hphi_lanczos_batch([H[0]] * 4, v2, 400, 1e-12)
    e = [r["e0"] for r in res]
    assert max(e) - min(e) < 1e-11 * abs(e[0])


def test_many_copies_fill_the_gpu():
    cfg = configs.heisenberg_chain16()
    m, b, h = pair(cfg["model"], 16, 8, 0, cfg["terms"])
    n = 2 * ctx().sm_count + 7
    vs = [torch.from_numpy(random_vectors(m.dim, 1, 100 + i)[:, 0]).cuda() for i in range(n)]
    res = hphi.hphi_lanczos_batch([h] * n, vs, 400, 1e-12, check_every=16)
    ref = -7.142296360616793  # dense / ARPACK value of the N=16 chain (pinned in the oracle tests)
    assert all(r["converged"] for r in res)
    assert max(abs(r["e0"] - ref) for r in res) < 1e-10 * abs(ref)


def test_edge_cases():
    cfg = configs.heisenberg_chain16()
    m, b, h = pair(cfg["model"], 16, 8, 0, cfg["terms"])
    # fully polarised sector: one state, H = sum Jz/4
    mp, bp, hp = pair("SPIN_HALF", 6, 6, 0, heisenberg_terms(chain(6), 1.3))
    # an eigenvector as start vector: invariant after one step
    m8, b8, h8 = pair("SPIN_HALF", 8, 4, 0, heisenberg_terms(chain(8), 1.0))
    E, U = np.linalg.eigh(O.dense_matrix(m8))
    vs = [torch.zeros(m.dim, dtype=torch.float64, device="cuda"),
          torch.from_numpy(random_vectors(m.dim, 1, 2)[:, 0]).cuda(),
          torch.ones(1, dtype=torch.float64, device="cuda"),
          torch.from_numpy(U[:, 0].copy()).cuda()]
    res = hphi.hphi_lanczos_batch([h, h, hp, h8], vs, 5, 1e-12, check_every=2)
    assert res[0]["status"] == -1                            # zero start vector
    assert res[1]["status"] == -4 and res[1]["steps"] == 5   # not converged in 5 steps
    assert res[2]["breakdown"] and res[2]["steps"] == 1 and abs(res[2]["e0"] - 6 * 1.3 / 4) < 1e-14
    assert res[3]["breakdown"] and res[3]["steps"] == 1 and abs(res[3]["e0"] - E[0]) < 1e-12
    with pytest.raises(ValueError):  # refused by the binding before any launch
        hphi.hphi_lanczos_batch([h], [torch.zeros(3, dtype=torch.float64, device="cuda")], 5, 1e-12)
    with pytest.raises(hphi.HphiError):  # refused by the library: FP64 only, checked before any launch
        opts_bad = hphi.hphi_lanczos_batch([h], [vs[1]], 0, 1e-12)
