"""Every device buffer of a simulator comes from the caller's allocator when one is given (here PyTorch's
caching allocator through sim_create_with_allocator): no direct cudaMalloc at create or while stepping
(pair lists grow on demand inside the step), the same trajectory as the default path, and every block
given back at destroy."""
import numpy as np
import pytest

from paper_2609_25653_b300 import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_torch_allocator_owns_every_device_buffer():
    from paper_2609_25653_b300 import ipcsim
    sc = scenes.fingertip_press(0, n_steps=6, pair_capacity=8)  # tiny initial pair list: it grows in the steps
    alloc = ipcsim.TorchAllocator()
    before = torch.cuda.memory_allocated()
    a = ipcsim.Simulator(sc, allocator=alloc)
    b = ipcsim.Simulator(sc)
    n_alloc, n_direct, held = a.memory()
    assert n_direct == 0 and n_alloc > 20 and held > 0
    assert torch.cuda.memory_allocated() - before >= held
    assert b.memory()[1] > 0 and b.memory()[0] == 0
    for k in range(5):
        sa, sb = a.step(), b.step()
        assert sa["status"] == 0 and sb["status"] == 0
        xa, xb = a.get_state()[0], b.get_state()[0]
        assert np.max(np.abs(xa - xb)) <= 1e-9 * a.L
    assert a.memory()[1] == 0 and a.memory()[0] >= n_alloc
    a.close()
    assert alloc.allocs == alloc.frees and not alloc.live


def test_torch_allocator_batch():
    from paper_2609_25653_b300 import ipcsim
    scs = [scenes.fingertip_press(s, n_steps=3) for s in (0, 1)]
    alloc = ipcsim.TorchAllocator()
    sim = ipcsim.Simulator.batch(scs, allocator=alloc)
    st = sim.step()
    assert st["status"] == 0 and sim.memory()[1] == 0
    sim.close()
    assert alloc.allocs == alloc.frees
