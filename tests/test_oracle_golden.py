"""The oracle's frequencies and bitstreams equal the digests stored in
tests/golden/oracle_digests.txt (written by make_oracle_digests.py). This
pins the oracle across compilers and CPU architectures (the GPU host is
AArch64, this one x86-64): IEEE FP32 with no contraction gives the same bits
on both."""
import os

from tests.golden import make_oracle_digests as mk


def test_oracle_digests_stable():
    path = os.path.join(os.path.dirname(os.path.abspath(mk.__file__)), "oracle_digests.txt")
    want = {}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        name, S, h_sf, h_w, nw = line.split()
        want[name] = (int(S), h_sf, h_w, int(nw))
    got = {name: (S, a, b, n) for name, S, a, b, n in mk.digests()}
    assert got == want
