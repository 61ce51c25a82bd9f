"""The Python binding's stream handling, on the host: a call given a stream runs with that
stream as torch's current one (so the device copies of its inputs, its outputs and the
library's work share it), and every binding call that stages tensors on the device does so."""

import inspect

from paper_2306_08967_gb300 import api

# calls with a stream argument that put no tensor on the device
NO_STAGING = {"step_array", "delete_nodes", "apply_edges_host", "ppr_refresh", "join"}


def test_stream_argument_becomes_the_current_stream(monkeypatch):
    seen = []

    class Ctx:
        def __init__(self, s):
            self.s = s

        def __enter__(self):
            seen.append(("enter", self.s))

        def __exit__(self, *exc):
            seen.append(("exit", self.s))

    monkeypatch.setattr(api.torch.cuda, "stream", Ctx)

    @api._on_stream
    def f(a, b=0, stream=None):
        seen.append(("run", stream))
        return a + b

    assert f(1) == 1 and seen == [("run", None)]
    seen.clear()
    assert f(1, 2, "S") == 3 and seen == [("enter", "S"), ("run", "S"), ("exit", "S")]
    seen.clear()
    assert f(1, stream="T") == 1 and seen == [("enter", "T"), ("run", "T"), ("exit", "T")]


def test_every_staging_call_is_wrapped():
    fns = [("batch_array", api.batch_array), ("core_svd", api.core_svd), ("apply_edges_multi", api.apply_edges_multi),
           ("step_multi", api.step_multi)]
    for cls in (api.DamfGraph, api.DamfFleet):
        for name, fn in inspect.getmembers(cls, predicate=inspect.isfunction):
            fns.append((name, fn))
        fns.append(("restore", api.DamfGraph.restore.__func__))
    checked = 0
    for name, fn in fns:
        if "stream" not in inspect.signature(fn).parameters or name in NO_STAGING:
            continue
        assert hasattr(fn, "__wrapped__"), name
        checked += 1
    assert checked >= 13
