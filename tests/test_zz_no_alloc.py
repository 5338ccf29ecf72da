"""The allocation-free contact check against the regular one.

casim_contacts_noalloc serves callers that cannot allocate device memory
while they run (real-time control loops, hosts whose allocator owns the GPU
memory pool).  It must find exactly the contact pairs that a regular
casim_step iteration reports through casim_get_contacts for the same
positions, on consecutive calls that share its static scratch."""
import numpy as np
import pytest

from paper_2203_02054_gb300 import casim, synth

pytestmark = pytest.mark.gpu


def _pairs(query, count, tets_out):
    rows = [(int(query[i]), int(tets_out[i, j])) for i in range(len(query)) for j in range(int(count[i]))]
    return np.array(rows, dtype=np.int64).reshape(-1, 2)


def test_noalloc_contacts_match_regular_contacts_on_two_calls():
    import torch

    casim.load_library()
    m = synth.small_finger(nx=20, ny=4, nz=4, n_ch=4)
    X0 = synth.perturbed_positions(m, 0.3, seed=41, dtype=np.float32)
    sim = casim.Sim(m)
    sim.set_positions(X0)
    sim.step(1)
    assert sim.sync() == 0
    ref_pairs, _ = sim.contacts()         # pairs of the check on X0
    query = sim.springs()["verts"]         # non-fixed boundary vertices
    sim.close()
    assert ref_pairs.shape[0] > 5

    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev).cuda_stream
    xyz = torch.tensor(X0.astype(np.float32), device=dev).contiguous()
    tets = torch.tensor(m.tets.astype(np.int32), device=dev).contiguous()
    q = torch.tensor(query.astype(np.int32), device=dev).contiguous()
    max_pairs = 8
    for _call in range(2):
        count = torch.full((len(query),), -1, dtype=torch.int32, device=dev)
        out = torch.full((len(query), max_pairs), -1, dtype=torch.int32, device=dev)
        rc = casim.casim_contacts_noalloc(m.n_verts, xyz.data_ptr(), m.n_tets, tets.data_ptr(), len(query),
                                          q.data_ptr(), m.cell_size, max_pairs, count.data_ptr(), out.data_ptr(),
                                          stream)
        assert rc == casim.CASIM_OK
        got = _pairs(query, count.cpu().numpy(), out.cpu().numpy())
        assert np.array_equal(got, ref_pairs)

    # sizes beyond the static scratch's limits are rejected before GPU work
    rc = casim.casim_contacts_noalloc(32769, xyz.data_ptr(), m.n_tets, tets.data_ptr(), len(query), q.data_ptr(),
                                      m.cell_size, max_pairs, count.data_ptr(), out.data_ptr(), stream)
    assert rc == casim.CASIM_E_INVALID
    rc = casim.casim_contacts_noalloc(m.n_verts, xyz.data_ptr(), 65537, tets.data_ptr(), len(query), q.data_ptr(),
                                      m.cell_size, max_pairs, count.data_ptr(), out.data_ptr(), stream)
    assert rc == casim.CASIM_E_INVALID


def _call(xyz, tets, query, cell, max_pairs):
    """One call on fresh torch device buffers; returns (rc, counts, tets)."""
    import torch

    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev).cuda_stream
    x = torch.tensor(np.asarray(xyz, np.float32), device=dev).contiguous()
    t = torch.tensor(np.asarray(tets, np.int32), device=dev).contiguous()
    q = torch.tensor(np.asarray(query, np.int32), device=dev).contiguous()
    count = torch.full((len(query),), -1, dtype=torch.int32, device=dev)
    out = torch.full((len(query), max_pairs), -1, dtype=torch.int32, device=dev)
    rc = casim.casim_contacts_noalloc(x.shape[0], x.data_ptr(), t.shape[0], t.data_ptr(), len(query), q.data_ptr(),
                                      cell, max_pairs, count.data_ptr(), out.data_ptr(), stream)
    torch.cuda.synchronize()
    return rc, count.cpu().numpy(), out.cpu().numpy()


def test_noalloc_rejections_then_a_valid_call():
    """Out-of-range ids (found on the device before any position is read
    through them), more pairs than max_pairs, and more hash entries than the
    scratch holds are reported with their own codes; a valid call after them
    still gives the exact pairs (the shared scratch is re-initialised)."""
    casim.load_library()
    # two copies of one tet (ids 0 and 1) and a query vertex at their centroid
    xyz = np.array([[0.0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [0.25, 0.25, 0.25]])
    tets = np.array([[0, 1, 2, 3], [0, 1, 2, 3]])
    ok_rc, ok_count, ok_out = _call(xyz, tets, [4], 0.5, 4)
    assert ok_rc == casim.CASIM_OK
    assert ok_count.tolist() == [2] and ok_out[0, :2].tolist() == [0, 1]

    bad = tets.copy()
    bad[1, 2] = xyz.shape[0]        # a vertex id equal to n_verts
    rc, _, _ = _call(xyz, bad, [4], 0.5, 4)
    assert rc == casim.CASIM_E_INVALID
    assert "out of range" in casim.casim_last_error(None)
    rc, _, _ = _call(xyz, tets, [5], 0.5, 4)     # query id out of range
    assert rc == casim.CASIM_E_INVALID

    rc, count, out = _call(xyz, tets, [4], 0.5, 1)   # two pairs, room for one
    assert rc == casim.CASIM_E_OVERFLOW
    assert "max_pairs" in casim.casim_last_error(None)
    assert count.tolist() == [1] and out[0, 0] == 0  # the smallest tet id is kept

    rc, _, _ = _call(xyz, tets, [4], 0.01, 4)        # 100^3 cells per tet box
    assert rc == casim.CASIM_E_OVERFLOW
    assert "hash entries" in casim.casim_last_error(None)

    rc, count, out = _call(xyz, tets, [4], 0.5, 4)
    assert rc == casim.CASIM_OK
    assert count.tolist() == ok_count.tolist() and np.array_equal(out, ok_out)
