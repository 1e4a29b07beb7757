"""Locate and load liblbm.so (placeholder until the C ABI lands)."""


class LbmError(RuntimeError):
    pass


def lib():
    raise LbmError("liblbm.so has not been built yet")
