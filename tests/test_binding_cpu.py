"""Without a GPU: the binding refuses host tensors where the library wants
device pointers, before it calls the library."""
import pytest

import paper_2109_05410_gb300 as ooc

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("call", [
    lambda u: ooc.ooc_heat7_steps(u, u.clone(), 1),
    lambda u: ooc.ooc_compress(u, 16),
    lambda u: ooc.ooc_wave25_steps(u, u.clone(), u.clone(), 1),
    lambda u: ooc.ooc_gather(u.flatten(), torch.zeros(2, dtype=torch.int64)),
    lambda u: ooc.ooc_bf16_pack(u),
])
def test_host_tensors_are_refused(call):
    ooc.build()
    u = torch.zeros((8, 8, 8), dtype=torch.float32)
    with pytest.raises(ValueError):
        call(u)
