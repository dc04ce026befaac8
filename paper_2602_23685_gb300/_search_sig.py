"""ctypes signatures of the search entry points (ALNS, BRKGA, serving)."""


def register(L):
    return L
