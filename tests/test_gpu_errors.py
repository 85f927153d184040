"""Error statuses from the GPU path (host-detected and device flags; no
kernel traps or hangs)."""
import pytest
import torch

from paper_cs_0702131_gb300 import synth
from paper_cs_0702131_gb300.aica import AicaError, Mesh

pytestmark = pytest.mark.gpu


def test_not_built_and_not_binned():
    c = synth.make("t0")
    m = Mesh(c["mesh"], c["box"])
    out = torch.empty((len(c["pos"]), 3), dtype=torch.float32, device="cuda")
    with pytest.raises(AicaError) as e:
        m.forces([1.0], [1.0], "fp32", out=out)
    assert e.value.name == "AICA_ERR_NOT_BUILT"
    m.build_lists(2.5)
    with pytest.raises(AicaError) as e:
        m.forces([1.0], [1.0], "fp32", out=out)
    assert e.value.name == "AICA_ERR_NOT_BUILT"


def test_bad_arguments():
    c = synth.make("t0")
    m = Mesh(c["mesh"], c["box"])
    with pytest.raises(AicaError) as e:
        m.build_lists(c["box"]["L"][0] * 0.6)          # rc + skin >= L/2
    assert e.value.name == "AICA_ERR_INVALID_ARG"
    m.build_lists(2.5)
    pos = torch.tensor(c["pos"], device="cuda")
    sp = torch.zeros(len(pos), dtype=torch.int32, device="cuda")
    sp[3] = 1
    m.bin(pos, sp)
    with pytest.raises(AicaError) as e:
        m.forces([1.0], [1.0], "fp32")                # species 1 with one species given
    assert e.value.name == "AICA_ERR_INVALID_ARG"
    sp[3] = 9
    with pytest.raises(AicaError) as e:
        m.bin(pos, sp)
    assert e.value.name == "AICA_ERR_INVALID_ARG"
