"""ctypes binding of libshouji.so (filled in with the C-ABI)."""
__all__ = []
