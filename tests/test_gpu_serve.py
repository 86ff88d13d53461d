"""Serving loop: a mixed stream of ground-state and spectrum requests gives,
for every request, the result the same request gives alone (bit for bit), the
oracle's energy, and the dense resolvent's D(z); memory admission queues
requests without changing results; the grid lane agrees with the block lane."""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import spectrum as S
from gpu_util import ctx, pair
from paper_2307_13222_gb300 import hphi
from workloads import chain, ladder, heisenberg_terms, hubbard_terms, uniform_couplings, random_vectors

pytestmark = pytest.mark.gpu

OMEGA = np.linspace(0.0, 4.0, 25)
ETA = 0.1


def _mix():
    """(name, oracle model, hamiltonian, kind, seed, q)"""
    out = []
    specs = [("chain12", "SPIN_HALF", 12, 6, 0, heisenberg_terms(chain(12), uniform_couplings(12, 0.5, 1.5, 1))),
             ("ladder5", "SPIN_HALF", 10, 5, 0, heisenberg_terms(ladder(5), 1.0)),
             ("chain10", "SPIN_HALF", 10, 5, 0, heisenberg_terms(chain(10), 1.0)),
             ("hub6", "HUBBARD", 6, 3, 3, hubbard_terms(6, chain(6), t=1.0, U=6.0))]
    hams = {}
    for name, model, N, nu, nd, terms in specs:
        hams[name] = pair(model, N, nu, nd, terms) + (N,)
    plan = [("chain12", 0, 3, 0.0), ("ladder5", 1, 4, np.pi), ("chain10", 1, 5, 2 * np.pi / 10),
            ("hub6", 0, 6, 0.0), ("chain12", 1, 7, 2 * 2 * np.pi / 12), ("hub6", 1, 8, 2 * np.pi / 6),
            ("chain10", 0, 9, 0.0), ("ladder5", 0, 10, 0.0)]
    for name, kind, seed, q in plan:
        m, b, h, N = hams[name]
        out.append((name, m, h, N, kind, seed, q))
    return out


def _run(server, items):
    ids = [server.submit(h, kind=kind, seed=seed, max_steps=600, tol=1e-10, q=q, eta=ETA, omega=OMEGA)
           for (name, m, h, N, kind, seed, q) in items]
    server.run_until_done(ids)
    return [server.result(i) for i in ids]


def test_mix_equals_alone_and_oracle():
    items = _mix()
    srv = hphi.Server(ctx(), 2e9, max_active=8, chunk=8)
    mixed = _run(srv, items)
    srv.close()
    for it, r in zip(items, mixed):
        name, m, h, N, kind, seed, q = it
        assert r["done"] and r["status"] == 0, (name, r)
        alone_srv = hphi.Server(ctx(), 2e9, chunk=5)
        a = _run(alone_srv, [it])[0]
        alone_srv.close()
        assert a["e0"] == r["e0"] and a["steps"] == r["steps"], name
        if kind == 1:
            assert np.array_equal(a["D"], r["D"]) and a["krylov_steps"] == r["krylov_steps"], name
        H = O.dense_matrix(m)
        E, U = np.linalg.eigh(H)
        assert abs(r["e0"] - E[0]) < 1e-10 * abs(E[0]), name
        if kind == 1:
            phi = m.sz_sum(U[:, 0], np.exp(1j * q * np.arange(N)))
            want = S.resolvent_dense(H, phi, E[0] + OMEGA + 1j * ETA)
            assert np.abs(r["D"] - want).max() < 1e-7 * max(np.abs(want).max(), 1e-12), name


def test_memory_admission_queues_without_changing_results():
    items = _mix()[:4]
    big = hphi.Server(ctx(), 2e9)
    ref = _run(big, items)
    big.close()
    # room for about one of these requests at a time (each needs 30-80 KB)
    small = hphi.Server(ctx(), 1e5, chunk=4)
    ids = [small.submit(h, kind=kind, seed=seed, max_steps=600, tol=1e-10, q=q, eta=ETA, omega=OMEGA)
           for (name, m, h, N, kind, seed, q) in items]
    queued_seen = 0
    for _ in range(100000):
        if all(small.result(i)["done"] for i in ids):
            break
        running, queued = small.step()
        queued_seen = max(queued_seen, queued)
    got = [small.result(i) for i in ids]
    small.close()
    assert queued_seen >= 1
    for r0, r1 in zip(ref, got):
        assert r0["e0"] == r1["e0"] and r0["steps"] == r1["steps"]
        if r0["D"] is not None:
            assert np.array_equal(r0["D"], r1["D"])


def test_grid_lane_agrees_with_block_lane():
    name, m, h, N, kind, seed, q = _mix()[2]   # chain10 spectrum
    blk = hphi.Server(ctx(), 2e9)
    a = _run(blk, [(name, m, h, N, kind, seed, q)])[0]
    blk.close()
    grd = hphi.Server(ctx(), 2e9, small_max_dim=16)   # every problem goes to the grid lane
    b = _run(grd, [(name, m, h, N, kind, seed, q)])[0]
    grd.close()
    assert a["lane"] == 0 and b["lane"] == 1 and b["status"] == 0
    assert abs(a["e0"] - b["e0"]) < 1e-11 * abs(a["e0"])
    assert np.abs(a["D"] - b["D"]).max() < 1e-7 * np.abs(a["D"]).max()


def test_grid_lane_fp32_storage_error_stated():
    """The grid lane with FP32 vectors (FP64 scalars): a ground state's energy
    is the FP64 Rayleigh quotient of its FP32 ground-state vector, within 1e-9
    of the dense ground energy; a spectrum's D(z) within FP32 accuracy of the
    dense resolvent."""
    terms = heisenberg_terms(chain(14), uniform_couplings(14, 0.5, 1.5, 3))
    m, b, h = pair("SPIN_HALF", 14, 7, 0, terms)
    H = O.dense_matrix(m)
    E, U = np.linalg.eigh(H)
    srv = hphi.Server(ctx(), 2e9, small_max_dim=16, grid_dtype="f32")
    ids = [srv.submit(h, kind=0, seed=11, max_steps=600, tol=1e-8),
           srv.submit(h, kind=1, seed=12, max_steps=600, tol=1e-5, q=2 * np.pi / 14, eta=ETA, omega=OMEGA)]
    srv.run_until_done(ids)
    g, s = srv.result(ids[0]), srv.result(ids[1])
    srv.close()
    assert g["status"] == 0 and g["lane"] == 1
    err = abs(g["e0"] - E[0]) / abs(E[0])
    assert err < 1e-9, err
    assert s["status"] == 0 and s["lane"] == 1
    phi = m.sz_sum(U[:, 0], np.exp(1j * (2 * np.pi / 14) * np.arange(14)))
    want = S.resolvent_dense(H, phi, s["e0"] + OMEGA + 1j * ETA)
    assert np.abs(s["D"] - want).max() < 2e-3 * np.abs(want).max()
    with pytest.raises(ValueError):
        hphi.Server(ctx(), 2e9, grid_dtype="f16")
