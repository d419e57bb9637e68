"""GB300 (sm_103a) implementation of the S3CMTF hot path: the per-nonzero SGD epoch of
sparse coupled Tucker matrix-tensor factorisation (Choi, Jang, Kang, arXiv 1708.08640).

Submodules are imported lazily so that the input generator (``synth``) can be used without
loading the CUDA library:

    from paper_1708_08640_gb300 import synth          # numpy only
    from paper_1708_08640_gb300.model import S3CMTF   # loads libs3cmtf.so
"""

__all__ = ["S3CMTF", "S3LossFn", "s3_loss", "synth", "build"]


def __getattr__(name):
    if name == "S3CMTF":
        from .model import S3CMTF
        return S3CMTF
    if name in ("S3LossFn", "s3_loss"):
        from . import autograd
        return getattr(autograd, name)
    if name in ("synth", "build", "model", "autograd"):
        import importlib
        return importlib.import_module("." + name, __name__)
    raise AttributeError(name)
