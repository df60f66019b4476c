"""bench.py's timed region on CPU (no GPU): a session handed the NULL stream
runs on a private stream of the library's (the C ABI's rule), which events on
the caller's stream do not order with, so the timed helper refuses a NULL
stream before it runs anything."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class _Stream:
    cuda_stream = 0


class _Session:
    def __init__(self):
        self.calls = []

    def run(self, n, sync=True):
        self.calls.append(("run", n, sync))
        return n

    def profile(self, on=True):
        self.calls.append(("profile", on))


def test_timed_session_refuses_the_null_stream():
    pytest.importorskip("torch")
    sys.path.insert(0, ROOT)
    import bench
    s = _Session()
    with pytest.raises(RuntimeError, match="non-NULL stream"):
        bench.timed_session(s, 3, 2, _Stream(), bench.Dist(1))
    assert s.calls == []
