"""GB300 (sm_103a) library for the 14-addition orthogonal approximate DCT of
Bayer & Cintra (arXiv 1702.00817): blockwise 8x8 transform, D^2-merged
quantisation, inverse and reconstruction as hand-written CUDA kernels behind a
C ABI (include/adct.h).  Importing the package loads nothing; the CUDA library
is loaded by the first Codec and must have been built (see _build.build)."""

__all__ = ["Codec", "Image", "make_quant", "AdctError", "ADCTFunction", "build"]


def build(force: bool = False) -> str:
    from . import _build
    return _build.build(force=force)


def __getattr__(name):
    if name in ("Codec", "Image", "make_quant", "AdctError", "butterfly_host",
                "ADCT_Q_NONE", "ADCT_Q_STEP", "ADCT_Q_ZONAL", "ADCT_Q_STEP_ZONAL"):
        from . import codec
        return getattr(codec, name)
    if name == "ADCTFunction":
        from . import autograd
        return autograd.ADCTFunction
    raise AttributeError(name)
