"""GB300-native peridynamics hot path (bond-based PMB with breaking, state-based
LPS, explicit step, tangent JVP/VJP) behind the C-ABI library ``libpd``.

``import paper_1806_06917_gb300`` loads nothing native; the binding
(``paper_1806_06917_gb300.pd``) loads ``libpd.so`` on first use and raises if it
is missing. ``paper_1806_06917_gb300.workloads`` holds the seeded input shapes.
"""
import importlib

__all__ = ["pd", "workloads"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(__name__ + "." + name)
    raise AttributeError(name)
