"""The Python binding refuses, before any library call, tensors the library would read through a
wrong pointer: CPU tensors on the device path, and record arrays of unequal lengths; the map stays
usable afterwards."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu


def test_binding_rejects_host_tensors_and_unequal_lengths():
    import torch

    import paper_2105_04419_gb300 as V
    m = V.Map(16, 16, 16, 4)
    with pytest.raises(ValueError):  # CPU tensors on the device path
        m.set_occupancy(torch.zeros((3, 3), dtype=torch.int32), torch.ones(3, dtype=torch.uint8))
    with pytest.raises(ValueError):  # 3 coordinates, 2 values (device)
        m.set_occupancy(torch.zeros((3, 3), dtype=torch.int32, device="cuda"),
                        torch.ones(2, dtype=torch.uint8, device="cuda"))
    with pytest.raises(ValueError):  # 3 coordinates, 2 values (host)
        m.set_occupancy(np.zeros((3, 3), np.int32), np.ones(2, np.uint8))
    with pytest.raises(ValueError):  # a CPU tensor of queries
        m.query(torch.zeros((3, 3), dtype=torch.int32))
    with pytest.raises(ValueError):  # brick coordinates on the CPU, masks on the device
        m.set_occupancy_bricks(torch.zeros((1, 3), dtype=torch.int32), torch.zeros((1, 8), dtype=torch.int64, device="cuda"))
    occ = np.zeros((16, 16, 16), np.uint8)
    occ[3, 4, 5] = 1
    m.set_occupancy(torch.tensor([[5, 4, 3]], dtype=torch.int32, device="cuda"),
                    torch.ones(1, dtype=torch.uint8, device="cuda"))
    m.global_()
    assert np.array_equal(m.export_dense(), O.edt_factorised(occ, 4))
    m.close()
