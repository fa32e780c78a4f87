def bind(L):
    return None
