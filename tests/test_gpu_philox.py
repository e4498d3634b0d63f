"""The device Philox4x32-10 (the walks' generator) against the generator's published known answers.

Walk replays compare the device walk with the oracle's, which use the same generator; this test pins the
device generator itself to the definition (Salmon, Moraes, Dror & Shaw 2011), independently of the oracle.
"""
import json
import os

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1909_11873_gb300 import build

    build.build()


def test_device_philox_known_answers():
    from paper_1909_11873_gb300 import gwl

    kat = json.load(open(os.path.join(HERE, "golden", "philox4x32_10_kat.json")))["vectors"]
    rec = [[int(x, 16) for x in v["counter"] + v["key"]] for v in kat]
    want = [[int(x, 16) for x in v["output"]] for v in kat]
    # words above 2^31 travel as their int32 bit patterns
    inp = torch.tensor([[w - (1 << 32) if w >= 1 << 31 else w for w in r] for r in rec], dtype=torch.int64).cuda()
    got = gwl.philox_eval(inp).cpu().tolist()
    assert got == want, [[hex(x) for x in g] for g in got]
