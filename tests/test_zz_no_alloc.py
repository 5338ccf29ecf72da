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
