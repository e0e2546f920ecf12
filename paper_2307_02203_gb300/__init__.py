"""GB300 (sm_103a) dependence volumes: Pearson and KSG mutual information between
a reference vertex and every vertex of an ensemble grid, behind the C ABI of
``libndf.so`` (declared in ``include/ndf.h``).

``paper_2307_02203_gb300.ndf`` is the ctypes binding; importing it raises
``ImportError`` when the library has not been built (there is no CPU fallback).
``paper_2307_02203_gb300.build`` compiles the library in-tree for sm_103a."""
import importlib


def __getattr__(name):
    if name == "ndf":
        return importlib.import_module(__name__ + ".ndf")
    raise AttributeError(name)
